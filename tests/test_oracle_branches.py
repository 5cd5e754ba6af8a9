"""Pins of the oracle's branch enumeration (admissible results of marginal decisions).

A float32 rasterizer may take a decision the other way when its FP64 value lies within
float32 rounding of the threshold (the 1/255 skip, the 1e-4 stop, the 0.99 clamp, sigma < 0,
a tile rectangle edge). ``oracle.render_leaves`` lists every composite reachable that way by
a depth-first walk; ``oracle.render_bwd_envelope`` bounds the adjoint over the leaves a test
admits; ``oracle.bin_ext`` adds the list members that a marginal projection decision could
add or remove. These tests pin them to things other than themselves: an exhaustive filter
over every assignment of every decision on tiny lists, the plain composite and adjoint when
no decision is marginal, the plain binning under each radius a marginal decision allows, and
the plain adjoint of each branch realised by nudging the input across its threshold. CPU only.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import scenes

M_REL, M_SIG = 1e-3, 1e-3
MARGINS = np.array([M_REL, 1e-4, 2e-6, 1e-6, M_SIG, 1e-6])


def one_pixel_projection(sig, opac, colors):
    """n splats over a 1x1 image (one 16x16 tile): splat k has exponent sig[k] at the pixel
    centre (mean one pixel to the right, conic a = 2 sigma), opacity opac[k], ascending depth."""
    n = len(sig)
    mean2d = np.tile([1.5, 0.5], (n, 1)).astype(float)
    conic = np.zeros((n, 3))
    conic[:, 0] = 2.0 * np.asarray(sig, float)
    conic[:, 2] = 1.0
    depth = np.arange(1, n + 1, dtype=float)
    radius = np.ones(n, np.int32)
    p = oracle.Projection(mean2d, conic, np.asarray(colors, float), np.asarray(opac, float), depth, radius,
                          np.tile([0, 0, 1, 1], (n, 1)).astype(np.int32), np.zeros(n, np.int32), radius.copy())
    return p


CAM1 = dict(viewmat=np.eye(4, dtype=np.float32), fx=1.0, fy=1.0, cx=0.5, cy=0.5, width=1, height=1,
            near=0.01, far=1e10)


def brute_force_outcomes(sig, opac, colors, unc):
    """Every assignment of an outcome to each of the five decisions of each pair (membership,
    sigma < 0, 0.99 clamp, 1/255 skip, 1e-4 stop), kept when every decision the walk
    evaluates either takes its FP64 outcome or is marginal there. Returns the distinct
    (C, T, n_contrib) and, for each, the contributor list (index, alpha, T before, G, clamped)."""
    n = len(sig)
    out = {}
    for assign in itertools.product(range(32), repeat=n):
        T, C, last, recs, ok = 1.0, np.zeros(3), 0, [], True
        stopped = False
        for i in range(n):
            bits = [(assign[i] >> k) & 1 for k in range(5)]  # 1 = the non-FP64 outcome

            def take(fp, marginal, bit):
                nonlocal ok
                if bit and not marginal:
                    ok = False
                return fp if not bit else (not fp)

            member = take(unc[i] != 1, unc[i] != 0, bits[0])
            if not ok:
                break
            if not member:
                continue
            s = sig[i]
            skip_sig = take(s < 0.0, abs(s) < M_SIG, bits[1])
            if not ok:
                break
            if skip_sig:
                continue
            G = np.exp(-s)
            araw = opac[i] * G
            clamped = take(araw >= 0.99, abs(araw - 0.99) < M_REL * 0.99, bits[2])
            if not ok:
                break
            a = 0.99 if clamped else araw
            skip_a = take(a < 1.0 / 255.0, abs(a * 255.0 - 1.0) < M_REL, bits[3])
            if not ok:
                break
            if skip_a:
                continue
            Tn = T * (1.0 - a)
            stop = take(Tn < 1e-4, abs(Tn - 1e-4) < M_REL * 1e-4, bits[4])
            if not ok:
                break
            if stop:
                stopped = True
                break
            C = C + np.asarray(colors[i]) * a * T
            recs.append((i, a, T, G, clamped))
            T, last = Tn, i + 1
        if not ok:
            continue
        key = (tuple(np.round(C, 12)), round(T, 12), last)
        out[key] = recs
        del stopped
    return out


def adjoint(recs, colors, sig, gC, bg=(0.0, 0.0, 0.0)):
    """Reverse-order adjoint of one contributor list (the textbook form; leaf 0's is pinned by
    finite differences elsewhere): per list position, d(u, v, a, b, c, opacity, r, g, b)."""
    n = len(colors)
    g = np.zeros((n, 12))
    B = np.array(bg, float)
    for (i, a, T, G, clamped) in reversed(recs):
        c = np.asarray(colors[i], float)
        g[i, 6:9] += a * T * gC
        dalpha = T * np.dot(c - B, gC)
        B = a * c + (1 - a) * B
        if clamped:
            continue
        g[i, 5] += dalpha * G
        dsig = -dalpha * a
        dx, dy = 1.0, 0.0  # mean one pixel right of the centre, same row
        a2 = 2.0 * sig[i]
        g[i, 2] += dsig * 0.5 * dx * dx
        g[i, 3] += dsig * dx * dy
        g[i, 4] += dsig * 0.5 * dy * dy
        g[i, 0] += dsig * (a2 * dx + 0.0 * dy)
        g[i, 1] += dsig * (0.0 * dx + 1.0 * dy)
    return g


def random_case(rng):
    """Three splats with decisions near their thresholds (each kind with some probability)."""
    kinds = rng.choice(["plain", "askip", "clamp", "sig", "opaque"], size=3)
    sig, opac = [], []
    for k in kinds:
        u = rng.uniform(-0.9, 0.9)
        if k == "plain":
            sig.append(rng.uniform(0.0, 2.0)); opac.append(rng.uniform(0.05, 0.9))
        elif k == "askip":
            sig.append(0.0); opac.append((1.0 / 255.0) * (1.0 + u * M_REL))
        elif k == "clamp":
            sig.append(0.0); opac.append(min(0.99 * (1.0 + u * M_REL), 1.0))
        elif k == "sig":
            sig.append(u * M_SIG); opac.append(rng.uniform(0.1, 0.9))
        else:  # clamped well past the margin
            sig.append(0.0); opac.append(0.995)
    # the last splat sometimes lands T (1 - alpha) near 1e-4
    T = 1.0
    for s, o in zip(sig[:2], opac[:2]):
        a = min(0.99, o * np.exp(-s))
        if s >= 0 and a >= 1 / 255:
            T *= 1 - a
    if rng.uniform() < 0.5 and 1e-4 / T < 0.5:
        sig[2] = 0.0
        opac[2] = 1.0 - 1e-4 * (1.0 + rng.uniform(-0.9, 0.9) * M_REL) / T
    colors = rng.uniform(0.05, 1.0, (3, 3))
    unc = [int(rng.choice([0, 0, 1, 2])) for _ in range(3)]
    return sig, opac, colors, unc


@pytest.mark.parametrize("seed", range(24))
def test_leaves_equal_exhaustive_filter(seed):
    rng = np.random.default_rng(seed)
    sig, opac, colors, unc = random_case(rng)
    p = one_pixel_projection(sig, opac, colors)
    eb = oracle.ExtBins(np.arange(3, dtype=np.int32), np.asarray(unc, np.uint8), np.array([0, 3], np.int32))
    lv = oracle.render_leaves(p, eb, CAM1, (16, 16), margins=MARGINS)
    n = int(lv.n[0, 0])
    assert n > 0
    got = {(tuple(np.round(lv.C[0, 0, l], 12)), round(float(lv.T[0, 0, l]), 12), int(lv.nc[0, 0, l]))
           for l in range(n)}
    want = brute_force_outcomes(sig, opac, colors, unc)
    assert got == set(want), (sig, opac, unc)
    # leaf 0 is the FP64 composite: every decision at its FP64 outcome, uncertain members as
    # the FP64 rectangle has them
    plain = oracle.render_fwd(p, np.array([i for i in range(3) if unc[i] != 1], np.int32),
                              np.array([0, sum(u != 1 for u in unc)], np.int32), CAM1, (16, 16))
    np.testing.assert_allclose(lv.C[0, 0, 0], plain.rgb[:, 0, 0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(10))
def test_envelope_is_min_max_over_admitted_leaves(seed):
    rng = np.random.default_rng(100 + seed)
    sig, opac, colors, unc = random_case(rng)
    p = one_pixel_projection(sig, opac, colors)
    eb = oracle.ExtBins(np.arange(3, dtype=np.int32), np.asarray(unc, np.uint8), np.array([0, 3], np.int32))
    lv = oracle.render_leaves(p, eb, CAM1, (16, 16), margins=MARGINS)
    n = int(lv.n[0, 0])
    outcomes = brute_force_outcomes(sig, opac, colors, unc)
    keys = [(tuple(np.round(lv.C[0, 0, l], 12)), round(float(lv.T[0, 0, l]), 12), int(lv.nc[0, 0, l]))
            for l in range(n)]
    # a key names one contributor list (two leaves share a key only when the same splats
    # contribute, e.g. a skip of the last pair and a stop there)
    gC = rng.standard_normal(3)
    dL = gC.reshape(3, 1, 1)
    masks = range(1, 1 << n) if n <= 5 else rng.integers(1, 1 << n, 24)
    for mask in masks:
        mask = int(mask)
        lo, hi, _ = oracle.render_bwd_envelope(p, eb, CAM1, dL, np.array([[mask]], np.uint64), (16, 16),
                                               margins=MARGINS)
        adj = []
        for l in range(n):
            if (mask >> l) & 1:
                adj.append(adjoint(outcomes[keys[l]], colors, sig, gC))
        adj = np.array(adj)
        np.testing.assert_allclose(lo, adj.min(axis=0), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(hi, adj.max(axis=0), rtol=1e-12, atol=1e-15)


def test_a_marginal_stop_alone_gives_both_outcomes():
    """Two clamped splats (alpha = 0.99, far from the clamp, sigma and 1/255 margins) bring
    T (1 - alpha) to 1e-4 within float rounding at the second one, whose only marginal decision
    is then the stop: the leaves are exactly the exhaustive filter's, the composite that blends
    it (and, past it, stops before the third) and the one that stops before it; the adjoint
    envelope over each is that list's textbook adjoint."""
    sig, opac = [0.002, 0.002, 0.5], [0.995, 0.995, 0.5]
    colors = np.array([[0.9, 0.1, 0.2], [0.3, 0.8, 0.5], [0.2, 0.4, 0.9]])
    unc = [0, 0, 0]
    p = one_pixel_projection(sig, opac, colors)
    eb = oracle.ExtBins(np.arange(3, dtype=np.int32), np.zeros(3, np.uint8), np.array([0, 3], np.int32))
    lv = oracle.render_leaves(p, eb, CAM1, (16, 16), margins=MARGINS)
    n = int(lv.n[0, 0])
    keys = [(tuple(np.round(lv.C[0, 0, l], 12)), round(float(lv.T[0, 0, l]), 12), int(lv.nc[0, 0, l]))
            for l in range(n)]
    want = brute_force_outcomes(sig, opac, colors, unc)
    assert n == 2 and set(keys) == set(want)
    assert sorted(int(lv.nc[0, 0, l]) for l in range(n)) == [1, 2]
    gC = np.array([0.7, -1.1, 0.4])
    for l in range(n):
        lo, hi, _ = oracle.render_bwd_envelope(p, eb, CAM1, gC.reshape(3, 1, 1), np.array([[1 << l]], np.uint64),
                                               (16, 16), margins=MARGINS)
        np.testing.assert_allclose(lo, adjoint(want[keys[l]], colors, sig, gC), rtol=1e-12, atol=1e-15)
        np.testing.assert_array_equal(lo, hi)


def test_single_leaf_envelope_with_clamped_pairs_is_the_plain_adjoint():
    """As below, with opacity logits raised by 6 so that most pixels composite clamped pairs
    (alpha = 0.99, whose opacity and exponent get no gradient): one leaf per pixel, and the
    envelope over it is exactly orc_render_bwd."""
    wl = scenes.small_scene()
    cam = wl.cameras[0].as_dict()
    g = oracle.set_dict(wl.sets[0])
    g["opacity_logits"] = g["opacity_logits"] + 6.0
    f = oracle.forward(g, cam, wl.tile)
    assert np.mean(f.proj.opacity[f.proj.radius > 0] >= 0.99) > 0.5
    eb = oracle.bin_ext(f.proj, cam, wl.tile)
    lv = oracle.render_leaves(f.proj, eb, cam, wl.tile)
    assert np.all(lv.n == 1)
    dL = np.random.default_rng(2).standard_normal((3, 128, 128))
    lo, hi, _ = oracle.render_bwd_envelope(f.proj, eb, cam, dL, np.ones((128, 128), np.uint64), wl.tile)
    want = oracle.render_bwd(f.proj, f.ids, f.tile_start, cam, dL, wl.tile)
    np.testing.assert_array_equal(lo, hi)
    for name, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                       ("color", slice(6, 9))]:
        np.testing.assert_allclose(lo[:, cols], getattr(want, name).reshape(len(lo), -1), rtol=1e-12, atol=1e-14)


def test_single_leaf_envelope_is_the_plain_adjoint():
    """Zero margins: one leaf per pixel, equal to the plain composite, and the envelope over it
    is exactly orc_render_bwd (lo = hi)."""
    wl = scenes.small_scene()
    cam = wl.cameras[0].as_dict()
    g = oracle.set_dict(wl.sets[0])
    f = oracle.forward(g, cam, wl.tile)
    eb = oracle.bin_ext(f.proj, cam, wl.tile)
    lv = oracle.render_leaves(f.proj, eb, cam, wl.tile)
    assert np.all(lv.n == 1)
    np.testing.assert_array_equal(lv.C[:, :, 0, :].transpose(2, 0, 1), f.image.rgb)
    np.testing.assert_array_equal(lv.T[:, :, 0], f.image.T_final)
    np.testing.assert_array_equal(lv.nc[:, :, 0], f.image.n_contrib)
    dL = np.random.default_rng(1).standard_normal((3, 128, 128))
    lo, hi, ab = oracle.render_bwd_envelope(f.proj, eb, cam, dL, np.ones((128, 128), np.uint64), wl.tile)
    want = oracle.render_bwd(f.proj, f.ids, f.tile_start, cam, dL, wl.tile)
    np.testing.assert_array_equal(lo, hi)
    for name, cols in [("mean2d", slice(0, 2)), ("conic", slice(2, 5)), ("opacity", slice(5, 6)),
                       ("color", slice(6, 9))]:
        np.testing.assert_allclose(lo[:, cols], getattr(want, name).reshape(len(lo), -1), rtol=1e-12, atol=1e-14)
    assert np.all(ab >= np.abs(lo) - 1e-15)


def test_each_branch_is_the_plain_result_of_an_input_across_the_threshold():
    """A splat whose alpha sits just above 1/255: leaf 0 includes it, leaf 1 skips it. Each
    equals the plain (margin-free) composite and adjoint of the same scene with that opacity
    moved by 1e-9 to the corresponding side of the threshold."""
    base_sig = [0.3, 0.0, 0.7]
    base_op = [0.4, (1 / 255) * (1 + 1e-6), 0.6]
    colors = np.array([[0.9, 0.1, 0.2], [0.3, 0.8, 0.5], [0.2, 0.4, 0.9]])
    p = one_pixel_projection(base_sig, base_op, colors)
    eb = oracle.ExtBins(np.arange(3, dtype=np.int32), np.zeros(3, np.uint8), np.array([0, 3], np.int32))
    lv = oracle.render_leaves(p, eb, CAM1, (16, 16), margins=MARGINS)
    assert lv.n[0, 0] == 2
    gC = np.array([0.7, -1.1, 0.4]).reshape(3, 1, 1)
    for leaf, nudge in ((0, 1 + 1e-9), (1, 1 - 1.2e-6)):
        q = one_pixel_projection(base_sig, [base_op[0], base_op[1] * nudge, base_op[2]], colors)
        ids, ts = np.arange(3, dtype=np.int32), np.array([0, 3], np.int32)
        img = oracle.render_fwd(q, ids, ts, CAM1, (16, 16))
        np.testing.assert_allclose(lv.C[0, 0, leaf], img.rgb[:, 0, 0], rtol=1e-7)
        want = oracle.render_bwd(q, ids, ts, CAM1, gC, (16, 16))
        lo, hi, _ = oracle.render_bwd_envelope(p, eb, CAM1, gC, np.array([[1 << leaf]], np.uint64), (16, 16),
                                               margins=MARGINS)
        np.testing.assert_allclose(lo[:, 6:9], want.color, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(lo[:, 5], want.opacity, rtol=1e-5, atol=1e-12)


def test_extended_lists_cover_every_allowed_radius():
    """A Gaussian with a marginal radius / rectangle decision may end up with radius r - 1, r
    or r + 1 on the GPU: the plain lists under each of those radii hold only members of the
    extended lists, and the certain members are in all three."""
    wl = scenes.small_scene()
    cam = wl.cameras[0].as_dict()
    g = oracle.set_dict(wl.sets[0])
    p = oracle.project(g, cam, wl.tile, margins=np.array([5e-4, 0.5, 2e-2, 2e-5, 1e-4, 2e-5]))
    flagged = (p.flags & (oracle.F_RADIUS | oracle.F_RECT)) != 0
    flagged &= (p.flags & oracle.F_GUARD) == 0
    assert flagged.sum() > 20
    eb = oracle.bin_ext(p, cam, wl.tile)
    gx, gy = oracle.grid(cam, wl.tile)
    members = {(t, int(i)) for t in range(gx * gy) for i in eb.ids[eb.tile_start[t]:eb.tile_start[t + 1]]}
    certain = {(t, int(i)) for t in range(gx * gy) for i, u in
               zip(eb.ids[eb.tile_start[t]:eb.tile_start[t + 1]], eb.unc[eb.tile_start[t]:eb.tile_start[t + 1]])
               if u == 0}
    for dr in (-1, 0, 1):
        q = oracle.Projection(p.mean2d, p.conic, p.color, p.opacity, p.depth,
                              np.where(flagged & (p.radius > 1), p.radius + dr, p.radius).astype(np.int32),
                              p.rect, p.flags, p.radius_all)
        ids, ts = oracle.bin_sort(q, cam, wl.tile)
        plain = {(t, int(i)) for t in range(gx * gy) for i in ids[ts[t]:ts[t + 1]]}
        assert plain <= members
        assert {m for m in certain} <= plain
    # the FP64 lists are exactly the members flagged as inside the FP64 rectangle
    ids, ts = oracle.bin_sort(p, cam, wl.tile)
    plain = {(t, int(i)) for t in range(gx * gy) for i in ids[ts[t]:ts[t + 1]]}
    inside = {(t, int(i)) for t in range(gx * gy) for i, u in
              zip(eb.ids[eb.tile_start[t]:eb.tile_start[t + 1]], eb.unc[eb.tile_start[t]:eb.tile_start[t + 1]])
              if u != 1}
    assert inside == plain


def test_a_marginal_guard_makes_every_tile_of_the_outer_rectangle_uncertain():
    """A Gaussian on the 1.3 x fov guard (|x/z| = 1.3 W / (2 fx) within the guard margin) may be
    culled or kept by a float32 projection: it is an uncertain member of every tile of its
    rectangle of radius r + 1 and a certain member of none, so the lists with it culled and
    with it kept are both admissible."""
    cam = dict(viewmat=np.eye(4, dtype=np.float32), fx=128.0, fy=128.0, cx=64.0, cy=64.0, width=128,
               height=128, near=0.01, far=1e10)
    z = 3.0
    g = dict(means=np.array([[0.65 * z, 0.0, z], [0.0, 0.0, z]]), log_scales=np.full((2, 3), -1.0),
             quats=np.tile([1.0, 0, 0, 0], (2, 1)), opacity_logits=np.zeros(2), sh=np.zeros((2, 16, 3)))
    p = oracle.project(g, cam, (16, 16), margins=np.array([5e-4, 0.5, 2e-2, 2e-5, 1e-4, 2e-5]))
    assert p.flags[0] & oracle.F_GUARD and p.radius_all[0] > 0
    eb = oracle.bin_ext(p, cam, (16, 16))
    gx, gy = oracle.grid(cam, (16, 16))
    r = p.radius_all[0] + 1
    u, v = p.mean2d[0]
    outer = [(tx, ty) for ty in range(gy) for tx in range(gx)
             if math.floor((u - r) / 16) <= tx < math.ceil((u + r) / 16) and math.floor((v - r) / 16) <= ty < math.ceil((v + r) / 16)]
    assert outer
    for tx, ty in outer:
        t = ty * gx + tx
        sl = slice(eb.tile_start[t], eb.tile_start[t + 1])
        k = list(eb.ids[sl]).index(0)  # a member of the tile...
        assert eb.unc[sl][k] != 0      # ...but never a certain one
