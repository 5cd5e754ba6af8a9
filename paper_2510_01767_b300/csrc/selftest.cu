// selftest.cu -- a self-test of the bounded device-side waits.
//
// Every spin of this library (the decoupled look-back of the scans and compactions) gives up
// after LB_SPIN_LIMIT polls, latches STATUS_TIMEOUT in the context's status word and lets its
// block carry on, so a wait that cannot end costs a few seconds and an error code instead of a
// hung GPU. This kernel makes one such wait run out on purpose: a single warp waits for the
// look-back word of a tile that no block ever publishes (an otherwise unused, zero word of the
// control block, polled under a tag that no launch uses). The host then reads the status.
#include "lookback.cuh"

namespace lobe {

__global__ void __launch_bounds__(32) k_selftest_wait(int *ctl)
{
    pdl_wait();
    // bytes 128..135 of the control block: never written (the status, generation and ticket
    // counters occupy its first 56 bytes), so the word stays 0, whose tag matches no launch
    const unsigned long long *slots = reinterpret_cast<const unsigned long long *>(ctl + 32);
    constexpr uint32_t NEVER = (1u << 30) - 1u;  // above every generation tag (< 2^30)
    const uint32_t sum = lb_exclusive_warp(slots, 1, NEVER, ctl);
    (void)sum;
}

cudaError_t launch_selftest_wait(int *ctl, cudaStream_t st)
{
    count_launch();
    launch_pdl(k_selftest_wait, dim3(1), dim3(32), 0, st, ctl);
    return cudaGetLastError();
}

}  // namespace lobe
