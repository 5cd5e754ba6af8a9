// project.cu -- EWA projection of 3D Gaussians (forward and adjoint), SH colour, culling,
// visibility cropping.
//
// One thread per (set, Gaussian); the thread loops over the items that render that set, so
// the Gaussian's 236 bytes of parameters are read from HBM once per set rather than once per
// view (the multi-view batches of a KD block share one Gaussian set), and the adjoint
// accumulates its per-view gradients in registers and writes each parameter once.
//
// Mathematics (the 3DGS rasterizer the paper trains with; appendix "3DGS Training"):
//   p_c = V mu + t; Sigma = R S S^T R^T (R from the normalised quaternion, S = diag(exp(log_s)))
//   J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]];  cov2d = J W Sigma W^T J^T + 0.3 I
//   conic = cov2d^-1; radius = ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det))
//   u = fx x/z + cx, v = fy y/z + cy; colour = max(0, SH(normalize(mu - campos)) + 0.5);
//   opacity = sigmoid(logit). Culled (radius 0): z outside [near, far] (z in double, Sec. 3.3
//   frustum culling), |x/z| or |y/z| beyond 1.3 tan(fov/2), det <= 0, empty tile rectangle,
//   crop_mask == 0 (visibility cropping, Sec. 3.3).
#include "lookback.cuh"

namespace lobe {

// Real SH normalisation constants sqrt((2l+1)/(4pi) (l-|m|)!/(l+|m|)!) * (sqrt 2 for m != 0),
// folded with the integer coefficients of the Cartesian polynomials (Condon-Shortley phase).
__constant__ float kSH[16] = {
    0.28209479177387814f,                                                  // l0: 1/(2 sqrt(pi))
    -0.48860251190291992f, 0.48860251190291992f, -0.48860251190291992f,   // l1: sqrt(3/(4pi)) * (-y, z, -x)
    1.0925484305920792f, -1.0925484305920792f, 0.31539156525252005f,      // l2: xy, yz, (2zz-xx-yy)
    -1.0925484305920792f, 0.54627421529603959f,                           //     xz, (xx-yy)
    -0.59004358992664352f, 2.8906114426405538f, -0.45704579946446572f,    // l3: y(3xx-yy), xyz, y(4zz-xx-yy)
    0.37317633259011540f, -0.45704579946446572f, 1.4453057213202769f,     //     z(2zz-3xx-3yy), x(4zz-xx-yy), z(xx-yy)
    -0.59004358992664352f};                                               //     x(xx-3yy)

// Basis polynomials (without the constant) and their gradients w.r.t. (x, y, z).
__device__ __forceinline__ void sh_poly(int deg, float x, float y, float z, float P[16])
{
    P[0] = 1.0f;
    if (deg < 1) return;
    P[1] = y; P[2] = z; P[3] = x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    P[4] = x * y; P[5] = y * z; P[6] = 2.0f * zz - xx - yy; P[7] = x * z; P[8] = xx - yy;
    if (deg < 3) return;
    P[9] = y * (3.0f * xx - yy);
    P[10] = x * y * z;
    P[11] = y * (4.0f * zz - xx - yy);
    P[12] = z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    P[13] = x * (4.0f * zz - xx - yy);
    P[14] = z * (xx - yy);
    P[15] = x * (xx - 3.0f * yy);
}

__device__ __forceinline__ void sh_poly_grad(int k, float x, float y, float z, float &gx, float &gy, float &gz)
{
    float xx = x * x, yy = y * y, zz = z * z;
    switch (k) {
    case 1: gx = 0; gy = 1; gz = 0; break;
    case 2: gx = 0; gy = 0; gz = 1; break;
    case 3: gx = 1; gy = 0; gz = 0; break;
    case 4: gx = y; gy = x; gz = 0; break;
    case 5: gx = 0; gy = z; gz = y; break;
    case 6: gx = -2 * x; gy = -2 * y; gz = 4 * z; break;
    case 7: gx = z; gy = 0; gz = x; break;
    case 8: gx = 2 * x; gy = -2 * y; gz = 0; break;
    case 9: gx = 6 * x * y; gy = 3 * xx - 3 * yy; gz = 0; break;
    case 10: gx = y * z; gy = x * z; gz = x * y; break;
    case 11: gx = -2 * x * y; gy = 4 * zz - xx - 3 * yy; gz = 8 * y * z; break;
    case 12: gx = -6 * x * z; gy = -6 * y * z; gz = 6 * zz - 3 * xx - 3 * yy; break;
    case 13: gx = 4 * zz - 3 * xx - yy; gy = -2 * x * y; gz = 8 * x * z; break;
    case 14: gx = 2 * x * z; gy = -2 * y * z; gz = xx - yy; break;
    case 15: gx = 3 * xx - 3 * yy; gy = -6 * x * y; gz = 0; break;
    default: gx = gy = gz = 0; break;
    }
}

struct World {
    float mx, my, mz;
    float qw, qx, qy, qz, qinv;  // normalised quaternion and 1/|q|
    float s[3];
    float Sig[6];  // 00 01 02 11 12 22
};

// Rotation matrix (row-major) of the unit quaternion (r, x, y, z).
__device__ __forceinline__ void rotation(float r, float x, float y, float z, float R[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - r * z);       R[2] = 2.f * (x * z + r * y);
    R[3] = 2.f * (x * y + r * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - r * x);
    R[6] = 2.f * (x * z - r * y);       R[7] = 2.f * (y * z + r * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ void load_world(const SetParams &S, long long g, World &w)
{
    w.mx = S.means[3 * g + 0];
    w.my = S.means[3 * g + 1];
    w.mz = S.means[3 * g + 2];
    float4 q = reinterpret_cast<const float4 *>(S.quats)[g];
    float qn = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    w.qinv = rsqrtf(qn);
    w.qw = q.x * w.qinv; w.qx = q.y * w.qinv; w.qy = q.z * w.qinv; w.qz = q.w * w.qinv;
    for (int i = 0; i < 3; ++i) w.s[i] = __expf(S.log_scales[3 * g + i]);
    float R[9];
    rotation(w.qw, w.qx, w.qy, w.qz, R);
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * w.s[j];
    w.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    w.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    w.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    w.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    w.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    w.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
}

// colour = max(0, raw). A clamped channel is stored as -0.0: it composites exactly like +0.0,
// and its sign bit carries the clamp decision to the adjoint (gradient passes iff raw >= 0).
__device__ __forceinline__ float clamp_color(float raw) { return raw < 0.f ? -0.0f : raw; }
__device__ __forceinline__ bool color_clamped(float stored) { return (__float_as_uint(stored) >> 31) != 0; }

// View direction n = normalize(mu - campos) and the SH basis polynomials at n (the forward and
// the adjoint call this one function).
__device__ __forceinline__ float view_basis(const World &w, const float campos[3], int deg, float n[3], float Pp[16])
{
    const float dx = w.mx - campos[0], dy = w.my - campos[1], dz = w.mz - campos[2];
    const float il = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(dz, dz))));
    n[0] = __fmul_rn(dx, il);
    n[1] = __fmul_rn(dy, il);
    n[2] = __fmul_rn(dz, il);
    sh_poly(deg, n[0], n[1], n[2], Pp);
    return il;
}

// One term of the raw colour sum_b k_b P_b sh_b,ch (channel by channel in ascending band order).
__device__ __forceinline__ float sh_term(int b, const float Pp[16], float coef, float acc)
{
    return fmaf(__fmul_rn(kSH[b], Pp[b]), coef, acc);
}

// Opacity of a logit.
__device__ __forceinline__ float opacity_of(float logit) { return 1.0f / (1.0f + __expf(-logit)); }

// Camera-dependent part of the projection. Returns false when culled.
struct Cam2D {
    float x, y, z;      // camera-space mean (z rounded from the double evaluation)
    double zd;
    float T0[3], T1[3]; // rows of J W
    float ST0[3], ST1[3];
    float c00, c01, c11;
    float ca, cb, cc;
    float u, v;
    int radius;
    int x0, y0, x1, y1;
};

__device__ __forceinline__ double depth_of(const ItemParams &I, const World &w)
{
    // ((V20 x + V21 y) + V22 z) + V23, each operation rounded in double
    double t = __dadd_rn(__dmul_rn(I.Vz[0], (double)w.mx), __dmul_rn(I.Vz[1], (double)w.my));
    t = __dadd_rn(t, __dmul_rn(I.Vz[2], (double)w.mz));
    return __dadd_rn(t, I.Vz[3]);
}

__device__ __forceinline__ bool project_cam(const BatchParams &P, const ItemParams &I, const World &w, Cam2D &c)
{
    c.zd = depth_of(I, w);
    if (!(c.zd >= I.near_plane && c.zd <= I.far_plane)) return false;
    const float *V = I.V;
    c.x = V[0] * w.mx + V[1] * w.my + V[2] * w.mz + V[3];
    c.y = V[4] * w.mx + V[5] * w.my + V[6] * w.mz + V[7];
    c.z = (float)c.zd;
    float iz = 1.0f / c.z;
    float tx = c.x * iz, ty = c.y * iz;
    if (fabsf(tx) > I.limx || fabsf(ty) > I.limy) return false;
    float j00 = I.fx * iz, j02 = -I.fx * tx * iz, j11 = I.fy * iz, j12 = -I.fy * ty * iz;
    for (int k = 0; k < 3; ++k) {
        c.T0[k] = j00 * V[k] + j02 * V[8 + k];
        c.T1[k] = j11 * V[4 + k] + j12 * V[8 + k];
    }
    const float *S = w.Sig;
    c.ST0[0] = S[0] * c.T0[0] + S[1] * c.T0[1] + S[2] * c.T0[2];
    c.ST0[1] = S[1] * c.T0[0] + S[3] * c.T0[1] + S[4] * c.T0[2];
    c.ST0[2] = S[2] * c.T0[0] + S[4] * c.T0[1] + S[5] * c.T0[2];
    c.ST1[0] = S[0] * c.T1[0] + S[1] * c.T1[1] + S[2] * c.T1[2];
    c.ST1[1] = S[1] * c.T1[0] + S[3] * c.T1[1] + S[4] * c.T1[2];
    c.ST1[2] = S[2] * c.T1[0] + S[4] * c.T1[1] + S[5] * c.T1[2];
    c.c00 = c.T0[0] * c.ST0[0] + c.T0[1] * c.ST0[1] + c.T0[2] * c.ST0[2] + 0.3f;
    c.c01 = c.T1[0] * c.ST0[0] + c.T1[1] * c.ST0[1] + c.T1[2] * c.ST0[2];
    c.c11 = c.T1[0] * c.ST1[0] + c.T1[1] * c.ST1[1] + c.T1[2] * c.ST1[2] + 0.3f;
    float det = c.c00 * c.c11 - c.c01 * c.c01;
    if (!(det > 0.0f)) return false;
    float idet = 1.0f / det;
    c.ca = c.c11 * idet;
    c.cb = -c.c01 * idet;
    c.cc = c.c00 * idet;
    float mid = 0.5f * (c.c00 + c.c11);
    float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
    c.radius = (int)ceilf(3.0f * sqrtf(lam));
    c.u = I.fx * tx + I.cx;
    c.v = I.fy * ty + I.cy;
    tile_rect(c.u, c.v, c.radius, P.tw, P.th, I.gx, I.gy, c.x0, c.y0, c.x1, c.y1);
    return c.radius > 0 && c.x1 > c.x0 && c.y1 > c.y0;
}

// --------------------------------------------------------------------------- forward
//
// Memory layout of the forward (B300): a warp takes 32 consecutive Gaussians. Their SH rows
// (192 contiguous bytes each, 6 KB for the warp) are copied once into shared memory by
// coalesced 16-byte asynchronous copies (cp.async: no registers, all in flight while the
// geometry is loaded and projected), swizzled so that the per-thread reads of every view fall
// in distinct banks; the per-view colour then costs shared-memory reads instead of 12 strided
// 16-byte global loads a view. A warp whose Gaussians span two sets (at most one warp per set
// boundary) copies per thread instead. Staging the 48-byte splat records for contiguous stores
// as well was measured slower (it limits the SM to 7 blocks).

constexpr int PF_THREADS = 128;
constexpr int PF_WARPS = PF_THREADS / 32;
// SH rows: 12 float4 each, chunk c of Gaussian i at c ^ ((i >> 1) & 3), so that each quarter
// warp's 16-byte reads of one chunk index (threads i .. i + 7) fall in 8 distinct 16-byte bank
// groups without padding; 24 KB a block, 8 blocks (32 warps) an SM at 64 registers.
constexpr int PF_ROW = 12;
__device__ __forceinline__ int pf_slot(int i, int c) { return i * PF_ROW + (c ^ ((i >> 1) & 3)); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__global__ void __launch_bounds__(PF_THREADS, 8) k_project_fwd(const __grid_constant__ BatchParams P,
                                                              float4 *__restrict__ splat, int *__restrict__ radius,
                                                              int *__restrict__ tiles)
{
    pdl_wait();
    __shared__ float4 s_sh[PF_WARPS][32 * PF_ROW];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long t = (long long)blockIdx.x * PF_THREADS + threadIdx.x;
    if (t - lane >= P.n_gauss) return;  // the whole warp is past the end
    const bool valid = t < P.n_gauss;
    const int s = valid ? set_of_gauss(P, t) : P.n_sets - 1;
    const SetParams &S = P.set[s];
    const long long g = t - S.gauss_off;
    const bool cropped = !valid || (S.crop != nullptr && S.crop[g] == 0);
    const unsigned need = __ballot_sync(0xffffffffu, !cropped);
    // one set for the whole warp (lanes past the end count as the last set): contiguous rows
    const bool one_set = __all_sync(0xffffffffu, s == __shfl_sync(0xffffffffu, s, 0));
    const int nb = (P.sh_degree + 1) * (P.sh_degree + 1);
    const int per = (3 * nb + 3) / 4;  // float4 chunks holding the used coefficients
    float4 *row = &s_sh[wp][0];  // this lane's chunks at pf_slot(lane, c)
    if (one_set) {
        // chunk f = lane + 32 r of the warp's 32 x 12: Gaussian f / 12, chunk f % 12
        const float4 *base = reinterpret_cast<const float4 *>(S.sh) + 12 * (g - lane);
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int f = lane + 32 * r, i = f / 12, c = f - 12 * i;
            if (c < per && ((need >> i) & 1u)) cp_async16(&s_sh[wp][pf_slot(i, c)], base + f);
        }
    } else if (!cropped) {
        const float4 *shg = reinterpret_cast<const float4 *>(S.sh + 48 * g);
        for (int c = 0; c < per; ++c) cp_async16(row + pf_slot(lane, c), shg + c);
    }
    World w;
    if (!cropped) load_world(S, g, w);
    cp_async_wait_all();
    __syncwarp();
    if (!valid) return;
    float opacity = 0.0f;
    bool first = true;
    for (int k = 0; k < S.item_count; ++k) {
        const ItemParams &I = P.item[P.set_items[S.item_begin + k]];
        const long long e = I.entry_off + g;
        Cam2D c;
        if (cropped || !project_cam(P, I, w, c)) {
            radius[e] = 0;
            tiles[e] = 0;
            continue;
        }
        if (first) {
            opacity = opacity_of(S.logits[g]);
            first = false;
        }
        float n[3], Pp[16];
        view_basis(w, I.campos, P.sh_degree, n, Pp);
        float col[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            if (4 * i >= 3 * nb) break;
            const float4 q = row[pf_slot(lane, i)];
            const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int idx = 4 * i + m, b = idx / 3;
                if (b < nb) col[idx % 3] = sh_term(b, Pp, qv[m], col[idx % 3]);
            }
        }
        float4 *o = splat + 3 * e;
        o[0] = make_float4(c.u, c.v, c.ca, c.cb);
        o[1] = make_float4(c.cc, opacity, clamp_color(col[0] + 0.5f), clamp_color(col[1] + 0.5f));
        o[2] = make_float4(clamp_color(col[2] + 0.5f), c.z, 0.f, 0.f);
        radius[e] = c.radius;
        tiles[e] = (c.x1 - c.x0) * (c.y1 - c.y0);
    }
}

// --------------------------------------------------------------------------- visibility crop

__global__ void __launch_bounds__(256) k_visibility(const __grid_constant__ BatchParams P)
{
    pdl_wait();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P.n_gauss) return;
    const int s = set_of_gauss(P, t);
    const SetParams &S = P.set[s];
    const long long g = t - S.gauss_off;
    World w;
    load_world(S, g, w);
    bool vis = false;
    for (int k = 0; k < S.item_count && !vis; ++k) {
        Cam2D c;
        vis = project_cam(P, P.item[P.set_items[S.item_begin + k]], w, c);
    }
    if (vis) S.vis_mask[g] = 1;
}

// --------------------------------------------------------------------------- backward
//
// Chain rule from dL/d(u, v, conic, colour, opacity) to (mu, log_s, q, logit, sh):
//   conic = cov^-1:  dL/dcov = -C Gs C,  Gs = [[da, db/2], [db/2, dc]]
//   cov = T Sigma T^T + 0.3 I, T = J W:  dL/dT = 2 H T Sigma,  dL/dSigma = T^T H T
//   J(p_c), (u, v)(p_c) -> dL/dp_c -> dL/dmu = W^T dL/dp_c
//   Sigma = M M^T, M = R diag(s): dL/dM = 2 dL/dSigma M; dL/ds_j = sum_i dM_ij R_ij; dL/dR = dM diag(s)
//   q -> R (normalised quaternion), then through the normalisation
//   colour = max(0, SH + 0.5): masked where the raw value is negative; the view direction
//   mu - campos carries a gradient to mu through the normalisation.
// The adjoint runs in two kernels. The first visits every Gaussian once: it appends each one
// that some item sees to a list and, unless accumulating, zeroes the gradients of the others.
// The second walks the list, so every lane of every warp does the chain rule
// (culled Gaussians, often most of a large set, cost no issue slots there). Per-view
// contributions to dL/dSigma (6 values), dL/dmu and dL/dlogit are summed in registers over the
// set's items, the 48 SH gradients in a padded shared-memory row per thread; the Sigma -> (s, q)
// step runs once per Gaussian. A block of the second kernel takes 64 listed Gaussians, stages
// their SH coefficients into shared memory (192 contiguous bytes per Gaussian) and writes their
// SH gradients back the same way.
// The fused variant (k_project_bwd_adam) ends in the Adam update of each listed Gaussian
// instead: parameters and moments are read and written where the gradients would have been
// written, and the gradients stay in registers and shared memory. Gaussians off the list keep
// parameters and moments (sparse Adam); for standard Adam the first kernel records who is seen
// and a zero-gradient Adam pass updates the others afterwards.

constexpr int PB_THREADS = 64;
constexpr int PB_ROW = 49;  // odd row stride: the per-thread rows fall in distinct banks

constexpr int PL_THREADS = 1024, PL_ITEMS = 4, PL_TILE = PL_THREADS * PL_ITEMS;  // 4096 Gaussians per tile

// List (ascending, so neighbours in the list share cache sectors) of the Gaussians some item
// sees, by a single-pass compaction with decoupled look-back; the last tile writes the count.
// Unless accumulating, the gradients of the other Gaussians are zeroed here.
__global__ void __launch_bounds__(PL_THREADS) k_project_bwd_list(const __grid_constant__ BatchParams P,
                                                                 const int *__restrict__ radius, int accumulate,
                                                                 uint32_t *__restrict__ list, uint32_t *__restrict__ count,
                                                                 LB lb)
{
    pdl_wait();
    __shared__ int s_tile;
    __shared__ uint32_t s_gen, s_prefix;
    __shared__ uint32_t s_warp[PL_THREADS / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int tk;
        uint32_t gen;
        lb_take(lb.ctl, lb.stage, true, tk, gen);  // opens this call's look-back generation
        s_tile = tk;
        s_gen = gen;
    }
    __syncthreads();
    const int tile = s_tile;
    const long long n = P.n_gauss;
    const long long ntiles = (n + PL_TILE - 1) / PL_TILE;
    if (tile >= (ntiles > 0 ? ntiles : 1)) return;
    const uint32_t tag = lb_tag(s_gen, lb.stage);
    const long long w0 = (long long)tile * PL_TILE + (long long)warp * (32 * PL_ITEMS);
    const unsigned lt = lanemask_lt();
    bool vis[PL_ITEMS];
    uint32_t rank[PL_ITEMS], carry = 0;
#pragma unroll
    for (int r = 0; r < PL_ITEMS; ++r) {
        const long long t = w0 + r * 32 + lane;
        vis[r] = false;
        if (t < n) {
            const int s = set_of_gauss(P, t);
            const SetParams &S = P.set[s];
            const long long g = t - S.gauss_off;
            for (int k = 0; k < S.item_count && !vis[r]; ++k)
                vis[r] = radius[P.item[P.set_items[S.item_begin + k]].entry_off + g] > 0;
            if (S.vis_mask != nullptr) S.vis_mask[g] = vis[r] ? 1 : 0;  // fused standard Adam: who is seen
            if (!vis[r] && !accumulate) {
                for (int i = 0; i < 3; ++i) {
                    S.g_means[3 * g + i] = 0.f;
                    S.g_log_scales[3 * g + i] = 0.f;
                }
                reinterpret_cast<float4 *>(S.g_quats)[g] = make_float4(0.f, 0.f, 0.f, 0.f);
                S.g_logits[g] = 0.f;
                float4 *d = reinterpret_cast<float4 *>(S.g_sh + 48 * g);
#pragma unroll
                for (int i = 0; i < 12; ++i) d[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, vis[r]);
        rank[r] = carry + __popc(m & lt);
        carry += __popc(m);
    }
    uint32_t wex;
    const uint32_t agg = block_exclusive_scan<PL_THREADS>(lane == 0 ? carry : 0u, wex, s_warp);
    wex = __shfl_sync(0xffffffffu, wex, 0);
    if (warp == 0) {
        unsigned long long *slot = lb.slots + tile;
        uint32_t prefix = 0;
        if (tile == 0) {
            if (lane == 0) lb_publish(slot, tag, LB_INC, agg);
        } else {
            if (lane == 0) lb_publish(slot, tag, LB_AGG, agg);
            prefix = lb_exclusive_warp(lb.slots, tile, tag, lb.ctl);
            if (lane == 0) lb_publish(slot, tag, LB_INC, prefix + agg);
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (tile == (ntiles > 0 ? ntiles - 1 : 0)) *count = prefix + agg;
        }
    }
    __syncthreads();
    const uint32_t base = s_prefix + wex;
#pragma unroll
    for (int r = 0; r < PL_ITEMS; ++r)
        if (vis[r]) list[base + rank[r]] = (uint32_t)(w0 + r * 32 + lane);
}

// ADAM: instead of writing the gradients, apply the Adam update of the Gaussian's set in
// place (A), so that a Gaussian's gradient never leaves the kernel (the sparse step: only
// listed Gaussians change).
template <bool ADAM>
__device__ __forceinline__ void project_bwd_body(const BatchParams &P, const float4 *__restrict__ splat,
                                                 const int *__restrict__ radius, const float4 *__restrict__ grad2d,
                                                 int accumulate, const uint32_t *__restrict__ list,
                                                 const uint32_t *__restrict__ count, const AdamBatch *A)
{
    pdl_wait();
    __shared__ float s_sh[PB_THREADS * PB_ROW];
    __shared__ float s_gsh[PB_THREADS * PB_ROW];
    __shared__ const float *s_src[PB_THREADS];  // the Gaussian's SH coefficients
    __shared__ float *s_dst[PB_THREADS];        // and its SH gradients (ADAM: its SH, updated in place)
    __shared__ float *s_m[ADAM ? PB_THREADS : 1], *s_v[ADAM ? PB_THREADS : 1];  // ADAM: its SH moments
    __shared__ int s_set[ADAM ? PB_THREADS : 1];                                  // ADAM: its set
    const uint32_t nv = *count;
    const long long b0 = (long long)blockIdx.x * PB_THREADS;
    if (b0 >= (long long)nv) return;
    const int nblk = (int)((long long)nv - b0 < PB_THREADS ? (long long)nv - b0 : PB_THREADS);
    const bool any = threadIdx.x < nblk;  // every listed Gaussian is seen by some item
    const long long t = any ? (long long)list[b0 + threadIdx.x] : 0;
    const int s = any ? set_of_gauss(P, t) : 0;
    const SetParams &S = P.set[s];
    const long long g = t - S.gauss_off;
    World w;
    unsigned seen = 0;  // bit k: item k of the set (k < 32) sees the Gaussian
    if (any) {
        load_world(S, g, w);  // in flight while the block stages its SH coefficients
        s_src[threadIdx.x] = S.sh + 48 * g;
        if constexpr (ADAM) {
            s_dst[threadIdx.x] = A->set[s].p[4] + 48 * g;
            s_m[threadIdx.x] = A->set[s].m[4] + 48 * g;
            s_v[threadIdx.x] = A->set[s].v[4] + 48 * g;
            s_set[threadIdx.x] = s;
        } else {
            s_dst[threadIdx.x] = S.g_sh + 48 * g;
        }
        // which of the first 32 items see it (their radii read together, one round trip per
        // four), then every seen entry's inputs toward L2, so that the per-item loop below waits
        // on L2 rather than on DRAM (culled entries' lines are not fetched)
        const int nk = S.item_count < 32 ? S.item_count : 32;
        for (int k0 = 0; k0 < nk; k0 += 4) {
            int r4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                r4[j] = k0 + j < nk ? radius[P.item[P.set_items[S.item_begin + k0 + j]].entry_off + g] : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) seen |= (r4[j] > 0 ? 1u : 0u) << (k0 + j);
        }
        for (unsigned m = seen; m; m &= m - 1) {
            const long long e = P.item[P.set_items[S.item_begin + __ffs(m) - 1]].entry_off + g;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(grad2d + 3 * e));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(grad2d + 3 * e + 2));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(splat + 3 * e + 1));
        }
        if constexpr (ADAM) {
            // this Gaussian's Adam state, toward L2 while the adjoint computes: the SH moments
            // (192 bytes each, at most three 128-byte lines) and the other arrays' entries
            const AdamSet &Z = A->set[s];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Z.m[4] + 48 * g + 32 * i));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Z.v[4] + 48 * g + 32 * i));
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int w = a < 2 ? 3 : a == 2 ? 4 : 1;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Z.p[a] + w * g));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Z.m[a] + w * g));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Z.v[a] + w * g));
            }
        }
    }
    float *gsh = s_gsh + threadIdx.x * PB_ROW;
    const float *shr = s_sh + threadIdx.x * PB_ROW;
#pragma unroll
    for (int i = 0; i < 48; ++i) gsh[i] = 0.f;
    __syncthreads();
    const int nb = (P.sh_degree + 1) * (P.sh_degree + 1);
    {
        // all loads first (no load waits on another), then the shared-memory stores
        const int per = (3 * nb + 3) / 4;  // float4 chunks holding the used coefficients
        const int total = nblk * per;       // <= 12 * PB_THREADS
        float4 q[12];
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int j = threadIdx.x + r * PB_THREADS;
            q[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < total) {
                const int gi = j / per, c = j - gi * per;
                q[r] = reinterpret_cast<const float4 *>(s_src[gi])[c];
            }
        }
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int j = threadIdx.x + r * PB_THREADS;
            if (j < total) {
                const int gi = j / per, c = j - gi * per;
                float *d = s_sh + gi * PB_ROW + 4 * c;
                d[0] = q[r].x; d[1] = q[r].y; d[2] = q[r].z; d[3] = q[r].w;
            }
        }
    }
    __syncthreads();
    float gmu[3] = {0.f, 0.f, 0.f};
    float gls[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f};
    float glogit = 0.f;
    float sd_acc = 0.f;
    int sd_cnt = 0;
    if (any) {
        float gSig[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < S.item_count; ++k) {
            const ItemParams &I = P.item[P.set_items[S.item_begin + k]];
            const long long e = I.entry_off + g;
            if (k < 32 ? !((seen >> k) & 1u) : radius[e] <= 0) continue;
            Cam2D c;
            project_cam(P, I, w, c);  // recompute the forward intermediates (visible by radius > 0)
            const float4 g0 = grad2d[3 * e + 0], g1 = grad2d[3 * e + 1], g2 = grad2d[3 * e + 2];
            const float du = g0.x, dv = g0.y, da = g0.z, db = g0.w, dc = g1.x, dop = g1.y;
            const float4 sp1 = splat[3 * e + 1];
            const float o = sp1.y;
            glogit += dop * o * (1.f - o);
            // ---- colour / SH. The forward's clamp decisions (sign bits of the stored colour)
            // mask the colour gradient: md_ch = dL/dcolour_ch where the channel was not clamped.
            // (Recomputing the opacity and the raw colours from the staged coefficients instead
            // of reading these 32 bytes a view was measured slower: 1.79 -> 1.89 ms.)
            const float md[3] = {color_clamped(sp1.z) ? 0.f : g1.z, color_clamped(sp1.w) ? 0.f : g1.w,
                                 color_clamped(splat[3 * e + 2].x) ? 0.f : g2.x};
            float nv[3], Pp[16];
            const float il = view_basis(w, I.campos, P.sh_degree, nv, Pp);
            const float nx = nv[0], ny = nv[1], nz = nv[2];
            // dL/dsh_b,ch = k_b P_b md_ch; the view direction n gets sum_b k_b grad P_b (sum_ch md_ch sh_b,ch)
            float dn[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int b = 0; b < 16; ++b) {
                if (b >= nb) break;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) gsh[3 * b + ch] += kSH[b] * Pp[b] * md[ch];
                if (b > 0) {
                    float ax, ay, az;
                    sh_poly_grad(b, nx, ny, nz, ax, ay, az);
                    const float f = kSH[b] * (md[0] * shr[3 * b] + md[1] * shr[3 * b + 1] + md[2] * shr[3 * b + 2]);
                    dn[0] += f * ax; dn[1] += f * ay; dn[2] += f * az;
                }
            }
            float ndn = nx * dn[0] + ny * dn[1] + nz * dn[2];
            gmu[0] += (dn[0] - nx * ndn) * il;
            gmu[1] += (dn[1] - ny * ndn) * il;
            gmu[2] += (dn[2] - nz * ndn) * il;
            // ---- conic -> cov2d
            const float ca = c.ca, cb = c.cb, cc = c.cc;
            const float hb = 0.5f * db;
            const float CG00 = ca * da + cb * hb, CG01 = ca * hb + cb * dc;
            const float CG10 = cb * da + cc * hb, CG11 = cb * hb + cc * dc;
            const float H00 = -(CG00 * ca + CG01 * cb);
            const float H01 = -(CG00 * cb + CG01 * cc);
            const float H11 = -(CG10 * cb + CG11 * cc);
            // ---- cov2d = T Sigma T^T
            float dT0[3], dT1[3];
            for (int i = 0; i < 3; ++i) {
                dT0[i] = 2.f * (H00 * c.ST0[i] + H01 * c.ST1[i]);
                dT1[i] = 2.f * (H01 * c.ST0[i] + H11 * c.ST1[i]);
            }
            // dSigma = H00 T0 T0^T + H01 (T0 T1^T + T1 T0^T) + H11 T1 T1^T
            {
                const float *a = c.T0, *b = c.T1;
                gSig[0] += H00 * a[0] * a[0] + 2.f * H01 * a[0] * b[0] + H11 * b[0] * b[0];
                gSig[1] += H00 * a[0] * a[1] + H01 * (a[0] * b[1] + b[0] * a[1]) + H11 * b[0] * b[1];
                gSig[2] += H00 * a[0] * a[2] + H01 * (a[0] * b[2] + b[0] * a[2]) + H11 * b[0] * b[2];
                gSig[3] += H00 * a[1] * a[1] + 2.f * H01 * a[1] * b[1] + H11 * b[1] * b[1];
                gSig[4] += H00 * a[1] * a[2] + H01 * (a[1] * b[2] + b[1] * a[2]) + H11 * b[1] * b[2];
                gSig[5] += H00 * a[2] * a[2] + 2.f * H01 * a[2] * b[2] + H11 * b[2] * b[2];
            }
            // ---- T = J W  ->  J entries
            const float *V = I.V;
            const float dJ00 = dT0[0] * V[0] + dT0[1] * V[1] + dT0[2] * V[2];
            const float dJ02 = dT0[0] * V[8] + dT0[1] * V[9] + dT0[2] * V[10];
            const float dJ11 = dT1[0] * V[4] + dT1[1] * V[5] + dT1[2] * V[6];
            const float dJ12 = dT1[0] * V[8] + dT1[1] * V[9] + dT1[2] * V[10];
            const float iz = 1.f / c.z, iz2 = iz * iz, iz3 = iz2 * iz;
            const float fx = I.fx, fy = I.fy;
            float dpx = du * fx * iz - dJ02 * fx * iz2;
            float dpy = dv * fy * iz - dJ12 * fy * iz2;
            float dpz = -du * fx * c.x * iz2 - dv * fy * c.y * iz2 - dJ00 * fx * iz2 + dJ02 * 2.f * fx * c.x * iz3 -
                        dJ11 * fy * iz2 + dJ12 * 2.f * fy * c.y * iz3;
            gmu[0] += V[0] * dpx + V[4] * dpy + V[8] * dpz;
            gmu[1] += V[1] * dpx + V[5] * dpy + V[9] * dpz;
            gmu[2] += V[2] * dpx + V[6] * dpy + V[10] * dpz;
            // ---- selective densification statistic (Sec. 3.3)
            if (w.mx >= I.lo[0] && w.mx < I.hi[0] && w.my >= I.lo[1] && w.my < I.hi[1] && w.mz >= I.lo[2] &&
                w.mz < I.hi[2]) {
                float a = du * 0.5f * (float)I.W, b = dv * 0.5f * (float)I.H;
                sd_acc += sqrtf(a * a + b * b);
                sd_cnt += 1;
            }
        }
        // ---- Sigma -> (log_s, q) once per Gaussian
        {
            // gSig holds the entries G_kl (k <= l) of the symmetric full-matrix gradient T^T H T
            float D[9] = {gSig[0], gSig[1], gSig[2], gSig[1], gSig[3], gSig[4], gSig[2], gSig[4], gSig[5]};
            float R[9];
            rotation(w.qw, w.qx, w.qy, w.qz, R);  // recomputed here rather than kept live over the views
            float M[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * w.s[j];
            float dM[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    dM[3 * i + j] = 2.f * (D[3 * i + 0] * M[0 + j] + D[3 * i + 1] * M[3 + j] + D[3 * i + 2] * M[6 + j]);
            float dR[9];
            for (int j = 0; j < 3; ++j) {
                float ds = dM[j] * R[j] + dM[3 + j] * R[3 + j] + dM[6 + j] * R[6 + j];
                gls[j] = ds * w.s[j];
                dR[j] = dM[j] * w.s[j];
                dR[3 + j] = dM[3 + j] * w.s[j];
                dR[6 + j] = dM[6 + j] * w.s[j];
            }
            const float r = w.qw, x = w.qx, y = w.qy, z = w.qz;
            float dqw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
            float dqx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - r * dR[5] + z * dR[6] + r * dR[7] -
                               2.f * x * dR[8]);
            float dqy = 2.f * (-2.f * y * dR[0] + x * dR[1] + r * dR[2] + x * dR[3] + z * dR[5] - r * dR[6] + z * dR[7] -
                               2.f * y * dR[8]);
            float dqz = 2.f * (-2.f * z * dR[0] - r * dR[1] + x * dR[2] + r * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                               x * dR[6] + y * dR[7]);
            float qd = r * dqw + x * dqx + y * dqy + z * dqz;
            gq[0] = (dqw - r * qd) * w.qinv;
            gq[1] = (dqx - x * qd) * w.qinv;
            gq[2] = (dqy - y * qd) * w.qinv;
            gq[3] = (dqz - z * qd) * w.qinv;
        }
    }
    // ---- write the per-Gaussian parameters
    if (ADAM && any) {
        const AdamSet &Z = A->set[s];
        const AdamK &k = A->k[s];
        // every load first (none waits on a store), then the updates and the stores
        float pm[3], mm[3], vm[3], pl[3], ml[3], vl[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            pm[i] = Z.p[0][3 * g + i]; mm[i] = Z.m[0][3 * g + i]; vm[i] = Z.v[0][3 * g + i];
            pl[i] = Z.p[1][3 * g + i]; ml[i] = Z.m[1][3 * g + i]; vl[i] = Z.v[1][3 * g + i];
        }
        float4 pq = reinterpret_cast<float4 *>(Z.p[2])[g], mq = reinterpret_cast<float4 *>(Z.m[2])[g],
               vq = reinterpret_cast<float4 *>(Z.v[2])[g];
        float po = Z.p[3][g], mo = Z.m[3][g], vo = Z.v[3][g];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            adam_step(k, k.ss[AG_MEANS], gmu[i], pm[i], mm[i], vm[i]);
            adam_step(k, k.ss[AG_LOG_SCALES], gls[i], pl[i], ml[i], vl[i]);
        }
        adam_step(k, k.ss[AG_QUATS], gq[0], pq.x, mq.x, vq.x);
        adam_step(k, k.ss[AG_QUATS], gq[1], pq.y, mq.y, vq.y);
        adam_step(k, k.ss[AG_QUATS], gq[2], pq.z, mq.z, vq.z);
        adam_step(k, k.ss[AG_QUATS], gq[3], pq.w, mq.w, vq.w);
        adam_step(k, k.ss[AG_OPACITY], glogit, po, mo, vo);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Z.p[0][3 * g + i] = pm[i]; Z.m[0][3 * g + i] = mm[i]; Z.v[0][3 * g + i] = vm[i];
            Z.p[1][3 * g + i] = pl[i]; Z.m[1][3 * g + i] = ml[i]; Z.v[1][3 * g + i] = vl[i];
        }
        reinterpret_cast<float4 *>(Z.p[2])[g] = pq;
        reinterpret_cast<float4 *>(Z.m[2])[g] = mq;
        reinterpret_cast<float4 *>(Z.v[2])[g] = vq;
        Z.p[3][g] = po; Z.m[3][g] = mo; Z.v[3][g] = vo;
        if (S.sd_acc != nullptr && sd_cnt > 0) {
            S.sd_acc[g] += sd_acc;
            S.sd_cnt[g] += sd_cnt;
        }
    } else if (any) {
        if (accumulate) {
            for (int i = 0; i < 3; ++i) {
                S.g_means[3 * g + i] += gmu[i];
                S.g_log_scales[3 * g + i] += gls[i];
            }
            float4 *gq4 = reinterpret_cast<float4 *>(S.g_quats) + g;
            float4 q = *gq4;
            *gq4 = make_float4(q.x + gq[0], q.y + gq[1], q.z + gq[2], q.w + gq[3]);
            S.g_logits[g] += glogit;
        } else {
            for (int i = 0; i < 3; ++i) {
                S.g_means[3 * g + i] = gmu[i];
                S.g_log_scales[3 * g + i] = gls[i];
            }
            reinterpret_cast<float4 *>(S.g_quats)[g] = make_float4(gq[0], gq[1], gq[2], gq[3]);
            S.g_logits[g] = glogit;
        }
        if (S.sd_acc != nullptr && sd_cnt > 0) {
            S.sd_acc[g] += sd_acc;
            S.sd_cnt[g] += sd_cnt;
        }
    }
    __syncthreads();
    if constexpr (ADAM) {
        // ---- Adam on the block's SH: 12 float4 per Gaussian, consecutive threads take
        // consecutive chunks of one Gaussian's 192 bytes; in two halves of 6 chunks a thread,
        // each with all its loads (parameter, m, v) issued before the first update
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4 P4[6], M4[6], V4[6];
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const int j = threadIdx.x + (6 * h + r) * PB_THREADS;
                if (j < nblk * 12) {
                    const int gi = j / 12, c = j - gi * 12;
                    P4[r] = reinterpret_cast<const float4 *>(s_dst[gi])[c];
                    M4[r] = reinterpret_cast<const float4 *>(s_m[gi])[c];
                    V4[r] = reinterpret_cast<const float4 *>(s_v[gi])[c];
                }
            }
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const int j = threadIdx.x + (6 * h + r) * PB_THREADS;
                if (j < nblk * 12) {
                    const int gi = j / 12, c = j - gi * 12;
                    const AdamK &k = A->k[s_set[gi]];
                    const float *gv = s_gsh + gi * PB_ROW + 4 * c;
                    // the first three floats of a Gaussian's 48 are its degree-0 band
                    const float sa = c == 0 ? k.ss[AG_SH_DC] : k.ss[AG_SH_REST];
                    adam_step(k, sa, gv[0], P4[r].x, M4[r].x, V4[r].x);
                    adam_step(k, sa, gv[1], P4[r].y, M4[r].y, V4[r].y);
                    adam_step(k, sa, gv[2], P4[r].z, M4[r].z, V4[r].z);
                    adam_step(k, k.ss[AG_SH_REST], gv[3], P4[r].w, M4[r].w, V4[r].w);
                    reinterpret_cast<float4 *>(s_dst[gi])[c] = P4[r];
                    reinterpret_cast<float4 *>(s_m[gi])[c] = M4[r];
                    reinterpret_cast<float4 *>(s_v[gi])[c] = V4[r];
                }
            }
        }
    } else {
        // ---- SH gradients of the block's Gaussians: 12 float4 per Gaussian, consecutive threads
        // take consecutive chunks of one Gaussian's 192 bytes
#pragma unroll
        for (int r = 0; r < 12; ++r) {
            const int j = threadIdx.x + r * PB_THREADS;  // float4 slot: Gaussian j / 12, chunk j % 12
            if (j >= nblk * 12) break;
            const int gi = j / 12, c = j - gi * 12;
            float4 *dst = reinterpret_cast<float4 *>(s_dst[gi]) + c;
            const float *v = s_gsh + gi * PB_ROW + 4 * c;
            float4 a = make_float4(v[0], v[1], v[2], v[3]);
            if (accumulate) {
                const float4 b = *dst;
                a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
            }
            *dst = a;
        }
    }
}

__global__ void __launch_bounds__(PB_THREADS, 8)
    k_project_bwd(const __grid_constant__ BatchParams P, const float4 *__restrict__ splat,
                  const int *__restrict__ radius, const float4 *__restrict__ grad2d, int accumulate,
                  const uint32_t *__restrict__ list, const uint32_t *__restrict__ count)
{
    project_bwd_body<false>(P, splat, radius, grad2d, accumulate, list, count, nullptr);
}

__global__ void __launch_bounds__(PB_THREADS, 8)
    k_project_bwd_adam(const __grid_constant__ BatchParams P, const float4 *__restrict__ splat,
                       const int *__restrict__ radius, const float4 *__restrict__ grad2d,
                       const uint32_t *__restrict__ list, const uint32_t *__restrict__ count,
                       const __grid_constant__ AdamBatch A)
{
    project_bwd_body<true>(P, splat, radius, grad2d, 1, list, count, &A);
}

// --------------------------------------------------------------------------- launchers

cudaError_t launch_project_fwd(const BatchParams &P, float *splat, int *radius, int *tiles, cudaStream_t st)
{
    if (P.n_gauss == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((P.n_gauss + PF_THREADS - 1) / PF_THREADS);
    count_launch();
    launch_pdl(k_project_fwd, dim3(blocks), dim3(PF_THREADS), 0, st, P, reinterpret_cast<float4 *>(splat), radius,
               tiles);
    return cudaGetLastError();
}

cudaError_t launch_visibility(const BatchParams &P, cudaStream_t st)
{
    if (P.n_gauss == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((P.n_gauss + 255) / 256);
    count_launch();
    launch_pdl(k_visibility, dim3(blocks), dim3(256), 0, st, P);
    return cudaGetLastError();
}

cudaError_t launch_project_bwd(const BatchParams &P, const float *splat, const int *radius, const float *grad2d,
                               int accumulate, uint32_t *list, uint32_t *count, unsigned long long *lb_slots, int *ctl,
                               cudaStream_t st, const AdamBatch *adam)
{
    if (P.n_gauss == 0) return cudaSuccess;
    count_launch(2);
    const unsigned lblocks = (unsigned)((P.n_gauss + PL_TILE - 1) / PL_TILE);
    launch_pdl(k_project_bwd_list, dim3(lblocks), dim3(PL_THREADS), 0, st, P, radius, accumulate, list, count,
                                                       LB{lb_slots, ctl, ST_PBWD_LIST});
    const unsigned blocks = (unsigned)((P.n_gauss + PB_THREADS - 1) / PB_THREADS);
    if (adam)
        launch_pdl(k_project_bwd_adam, dim3(blocks), dim3(PB_THREADS), 0, st, P, reinterpret_cast<const float4 *>(splat),
                   radius, reinterpret_cast<const float4 *>(grad2d), list, count, *adam);
    else
        launch_pdl(k_project_bwd, dim3(blocks), dim3(PB_THREADS), 0, st, P, reinterpret_cast<const float4 *>(splat),
                   radius, reinterpret_cast<const float4 *>(grad2d), accumulate, list, count);
    return cudaGetLastError();
}

}  // namespace lobe
