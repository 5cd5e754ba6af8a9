"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a closed form, a library routine, an invariant that
the compositing equation implies, an independent brute-force formulation, or central
finite differences, so that a dropped term, a wrong sign, a swapped index or a transposed
operand in ``oracle/lobe_oracle.c`` fails at least one of them. CPU only.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle
import scenes

CAM128 = dict(viewmat=np.eye(4, dtype=np.float32), fx=128.0, fy=128.0, cx=64.0, cy=64.0,
              width=128, height=128, near=0.01, far=1e10)


def one_gaussian(mu, log_s, quat=(1, 0, 0, 0), logit=0.0, dc=(1.0, 1.0, 1.0)):
    sh = np.zeros((1, 16, 3))
    sh[0, 0] = dc
    return dict(means=np.array([mu], float), log_scales=np.array([log_s], float),
                quats=np.array([quat], float), opacity_logits=np.array([logit], float), sh=sh)


def unit_dirs(n, seed=0):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


# ----------------------------------------------------------------------------- SH

def real_sh_scipy(l, m, d):
    """Real SH with the Condon-Shortley phase from scipy's complex SH (library routine):
    Y_{l,m} = sqrt(2) Re Y_l^m (m>0), sqrt(2) Im Y_l^|m| (m<0), Y_l^0 (m=0)."""
    theta = np.arccos(np.clip(d[:, 2], -1, 1))  # polar
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = sps.sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return math.sqrt(2) * Y.real
    if m < 0:
        return math.sqrt(2) * Y.imag
    return Y.real


def test_sh_matches_scipy():
    d = unit_dirs(200)
    Y, _ = oracle.sh_basis(d)
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, k], real_sh_scipy(l, m, d), atol=1e-13, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_textbook_closed_forms():
    """A few real SH written out from the standard table (Condon-Shortley phase)."""
    d = unit_dirs(50, 1)
    x, y, z = d.T
    Y, _ = oracle.sh_basis(d)
    pi = math.pi
    np.testing.assert_allclose(Y[:, 0], 0.5 / math.sqrt(pi) * np.ones_like(x), atol=1e-14)
    np.testing.assert_allclose(Y[:, 1], -math.sqrt(3 / (4 * pi)) * y, atol=1e-14)
    np.testing.assert_allclose(Y[:, 2], math.sqrt(3 / (4 * pi)) * z, atol=1e-14)
    np.testing.assert_allclose(Y[:, 3], -math.sqrt(3 / (4 * pi)) * x, atol=1e-14)
    np.testing.assert_allclose(Y[:, 4], 0.5 * math.sqrt(15 / pi) * x * y, atol=1e-14)
    np.testing.assert_allclose(Y[:, 6], 0.25 * math.sqrt(5 / pi) * (3 * z * z - 1), atol=1e-14)
    np.testing.assert_allclose(Y[:, 8], 0.25 * math.sqrt(15 / pi) * (x * x - y * y), atol=1e-14)
    np.testing.assert_allclose(Y[:, 9], -0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y), atol=1e-13)
    np.testing.assert_allclose(Y[:, 12], 0.25 * math.sqrt(7 / pi) * z * (5 * z * z - 3), atol=1e-13)


def test_sh_orthonormal_by_quadrature():
    nodes, weights = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phis = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(nodes, phis, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (weights[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).reshape(-1)
    Y, _ = oracle.sh_basis(d)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_gradient_tangential_matches_fd():
    d = unit_dirs(20, 3)
    Y, dY = oracle.sh_basis(d)
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        Yp, _ = oracle.sh_basis(d + e)
        Ym, _ = oracle.sh_basis(d - e)
        np.testing.assert_allclose(dY[:, :, i], (Yp - Ym) / (2 * h), atol=1e-8)


def test_degree0_colour_is_constant():
    g = one_gaussian((0.1, -0.2, 3.0), (-2, -2, -2), dc=(0.3, -0.4, 1.0))
    for deg in (0, 3):
        p = oracle.project(g, CAM128, sh_degree=deg)
        want = np.maximum(0.0, 0.5 / math.sqrt(math.pi) * np.array([0.3, -0.4, 1.0]) + 0.5)
        np.testing.assert_allclose(p.color[0], want, atol=1e-15)


# ----------------------------------------------------------------------------- projection

def test_isotropic_on_axis_closed_form():
    s, z = 0.05, 4.0
    g = one_gaussian((0, 0, z), (math.log(s),) * 3, quat=(0.3, -0.5, 0.7, 0.2), logit=0.4)
    p = oracle.project(g, CAM128)
    var = (128 * s / z) ** 2 + 0.3
    np.testing.assert_allclose(p.mean2d[0], [64.0, 64.0], atol=1e-12)
    np.testing.assert_allclose(p.conic[0], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-15)
    assert p.radius[0] == math.ceil(3 * math.sqrt(var))
    # footprint pixel by pixel
    f = oracle.forward(g, CAM128)
    o = 1 / (1 + math.exp(-0.4))
    c = 0.5 / math.sqrt(math.pi) + 0.5
    ys, xs = np.mgrid[0:128, 0:128]
    rho2 = (xs + 0.5 - 64) ** 2 + (ys + 0.5 - 64) ** 2
    alpha = np.minimum(0.99, o * np.exp(-rho2 / (2 * var)))
    r = p.radius[0]
    tx0, tx1 = math.floor((64 - r) / 16), math.ceil((64 + r) / 16)
    inrect = (xs // 16 >= tx0) & (xs // 16 < tx1) & (ys // 16 >= tx0) & (ys // 16 < tx1)
    want = np.where(inrect & (alpha >= 1 / 255), c * alpha, 0.0)
    np.testing.assert_allclose(f.image.rgb[0], want, atol=1e-14)
    np.testing.assert_allclose(f.image.T_final, np.where(inrect & (alpha >= 1 / 255), 1 - alpha, 1.0), atol=1e-14)


def pinhole_uv(pc, fx=128.0, fy=128.0, cx=64.0, cy=64.0):
    return np.array([fx * pc[0] / pc[2] + cx, fy * pc[1] / pc[2] + cy])


def test_off_axis_cov2d_equals_numerical_jacobian():
    """cov2d = J Sigma J^T + 0.3 I with J the Jacobian of the pinhole map, here taken by
    central differences of (u, v)(x, y, z) -- an independent route to J."""
    mu = np.array([0.7, -0.4, 3.0])
    s = np.array([0.05, 0.11, 0.08])
    g = one_gaussian(mu, np.log(s))
    p = oracle.project(g, CAM128)
    J = np.zeros((2, 3))
    h = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        J[:, i] = (pinhole_uv(mu + e) - pinhole_uv(mu - e)) / (2 * h)
    cov = J @ np.diag(s ** 2) @ J.T + 0.3 * np.eye(2)
    conic = np.linalg.inv(cov)
    np.testing.assert_allclose(p.conic[0], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-8)
    np.testing.assert_allclose(p.mean2d[0], pinhole_uv(mu), atol=1e-12)


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_rotation_about_optical_axis_rotates_conic():
    q0 = np.array([0.9, 0.1, -0.3, 0.2])
    q0 /= np.linalg.norm(q0)
    ls = np.log([0.04, 0.12, 0.07])
    p0 = oracle.project(one_gaussian((0, 0, 3.0), ls, q0), CAM128)
    th = 0.7
    rz = np.array([math.cos(th / 2), 0, 0, math.sin(th / 2)])
    p1 = oracle.project(one_gaussian((0, 0, 3.0), ls, quat_mul(rz, q0)), CAM128)
    a, b, c = p0.conic[0]
    C0 = np.array([[a, b], [b, c]])
    R2 = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    # cov rotates as R cov R^T, and so does its inverse; the 0.3 I dilation is rotation invariant
    C1 = R2 @ C0 @ R2.T
    a1, b1, c1 = p1.conic[0]
    np.testing.assert_allclose([a1, b1, c1], [C1[0, 0], C1[0, 1], C1[1, 1]], rtol=1e-10, atol=1e-14)


def test_culling_rules():
    cam = dict(CAM128)
    mus = [(0, 0, 0.005),      # in front of the camera but nearer than the near plane
           (0, 0, -2.0),       # behind
           (0.7 * 3, 0, 3.0),  # |x/z| = 0.7 > 1.3*64/128 = 0.65: outside the guard
           (0.52 * 3, 0, 3.0),  # inside the guard, footprint reaches the image
           (0, 0, 3.0)]
    g = dict(means=np.array(mus, float), log_scales=np.full((5, 3), -3.0), quats=np.tile([1.0, 0, 0, 0], (5, 1)),
             opacity_logits=np.zeros(5), sh=np.zeros((5, 16, 3)))
    p = oracle.project(g, cam)
    assert list(p.radius > 0) == [False, False, False, True, True]
    crop = np.array([1, 1, 1, 1, 0], np.uint8)
    p2 = oracle.project(g, cam, crop=crop)
    assert list(p2.radius > 0) == [False, False, False, True, False]
    mask = oracle.visibility_crop(g, [cam])
    assert list(mask) == [0, 0, 0, 1, 1]


def test_visibility_crop_is_the_union_over_the_block_cameras():
    """Visibility cropping keeps a Gaussian that any camera of the block sees (Sec. 3.3): two
    cameras looking along +z and -z from the origin each see only the Gaussians in front of
    them, and the crop over both keeps all of them, whatever the order of the cameras."""
    mus = [(0, 0, 3.0), (0, 0, -3.0), (0.2, 0.1, 4.0), (-0.1, 0.2, -5.0)]
    g = dict(means=np.array(mus, float), log_scales=np.full((4, 3), -3.0), quats=np.tile([1.0, 0, 0, 0], (4, 1)),
             opacity_logits=np.zeros(4), sh=np.zeros((4, 16, 3)))
    back = dict(CAM128, viewmat=np.diag([1.0, -1.0, -1.0, 1.0]))  # a half turn about x: looks along -z
    assert list(oracle.visibility_crop(g, [CAM128])) == [1, 0, 1, 0]
    assert list(oracle.visibility_crop(g, [back])) == [0, 1, 0, 1]
    assert list(oracle.visibility_crop(g, [CAM128, back])) == [1, 1, 1, 1]
    assert list(oracle.visibility_crop(g, [back, CAM128])) == [1, 1, 1, 1]


def test_depth_key_is_float32_z():
    g = one_gaussian((0.1, 0.2, 3.3), (-3, -3, -3))
    vm = scenes.look_at((1.0, -2.0, 0.5), (0.0, 0.0, 4.0), up=(0, -1, 0))
    cam = dict(CAM128, viewmat=vm)
    p = oracle.project(g, cam)
    V = vm.astype(np.float64)
    z = ((V[2, 0] * 0.1 + V[2, 1] * 0.2) + V[2, 2] * 3.3) + V[2, 3]
    assert p.depth[0] == z
    assert oracle.depth_key(z) == np.float32(z).view(np.uint32)


# ----------------------------------------------------------------------------- compositing

def test_zero_opacity_gives_background():
    wl = scenes.small_scene(n=200)
    g = oracle.set_dict(wl.sets[0])
    g["opacity_logits"][:] = -800.0  # sigmoid -> 0 exactly in double
    bg = (0.2, 0.3, 0.4)
    f = oracle.forward(g, CAM128, bg=bg)
    for ch in range(3):
        assert np.all(f.image.rgb[ch] == bg[ch])
    assert np.all(f.image.T_final == 1.0)
    assert np.all(f.image.n_contrib == 0)


def test_weights_and_transmittance_sum_to_one():
    wl = scenes.small_scene()
    g = oracle.set_dict(wl.sets[0])
    f = oracle.forward(g, CAM128)
    np.testing.assert_allclose(f.image.wsum + f.image.T_final, 1.0, atol=1e-12)
    assert np.all(f.image.T_final >= 1e-4) and np.all(f.image.T_final <= 1.0)
    # transmittance is non-increasing along the list: dropping the back half of every list
    # (render a subset of Gaussians with larger depth removed) cannot lower T
    keep = g["means"][:, 2] < 4.0
    g2 = {k: v[keep] for k, v in g.items()}
    f2 = oracle.forward(g2, CAM128)
    assert np.all(f2.image.T_final >= f.image.T_final - 1e-15)


def test_permutation_invariance():
    wl = scenes.small_scene(n=300)
    g = oracle.set_dict(wl.sets[0])
    f = oracle.forward(g, CAM128)
    perm = np.random.default_rng(5).permutation(300)
    gp = {k: v[perm] for k, v in g.items()}
    fp = oracle.forward(gp, CAM128)
    np.testing.assert_array_equal(fp.image.rgb, f.image.rgb)
    np.testing.assert_array_equal(fp.image.T_final, f.image.T_final)


def test_opaque_front_gaussian_bounds_what_is_behind():
    wl = scenes.small_scene(n=300)
    g = oracle.set_dict(wl.sets[0])
    front = one_gaussian((0, 0, 1.0), (-1.5, -1.5, -1.5), logit=12.0, dc=(0.0, 0.0, 0.0))
    gg = {k: np.concatenate([front[k], g[k]]) for k in g}
    f = oracle.forward(gg, CAM128)
    # pixel at the optical axis: the front Gaussian has alpha clamped at 0.99 and colour 0.5
    c = f.image.rgb[:, 63, 63]
    assert np.all(c >= 0.99 * 0.5 - 1e-12)
    assert np.all(c <= 0.99 * 0.5 + 0.01 * max(1.0, g["sh"][:, 0].max()) + 1e-12)


def test_sort_matches_lexsort():
    wl = scenes.small_scene()
    g = oracle.set_dict(wl.sets[0])
    p = oracle.project(g, CAM128)
    ids, ts = oracle.bin_sort(p, CAM128)
    tiles, keys, gid = [], [], []
    for i in np.nonzero(p.radius > 0)[0]:
        r = p.rect[i]
        for ty in range(r[1], r[3]):
            for tx in range(r[0], r[2]):
                tiles.append(ty * 8 + tx)
                keys.append(np.float32(p.depth[i]).view(np.uint32))
                gid.append(i)
    tiles, keys, gid = map(np.array, (tiles, keys, gid))
    order = np.lexsort((gid, keys, tiles))
    np.testing.assert_array_equal(ids, gid[order])
    np.testing.assert_array_equal(ts, np.searchsorted(tiles[order], np.arange(65), side="left"))


def test_tiled_equals_bruteforce_membership():
    """Tiled lists from the global sort == per-pixel gather of all Gaussians whose tile
    rectangle holds the pixel's tile, sorted by depth (no keys, no ranges)."""
    wl = scenes.small_scene()
    g = oracle.set_dict(wl.sets[0])
    f = oracle.forward(g, CAM128)
    rgb, T, _ = oracle.render_untiled(f.proj, CAM128, respect_rect=True)
    np.testing.assert_array_equal(rgb, f.image.rgb)
    np.testing.assert_array_equal(T, f.image.T_final)


@pytest.mark.parametrize("n", [64, 1000])
def test_tiled_equals_untiled_without_truncation(n):
    """With every opacity below 0.35 a Gaussian has alpha < 1/255 at any pixel outside its
    3-sigma tile rectangle, so tiling changes nothing: the tiled image equals plain per-pixel
    compositing of *all* Gaussians sorted by depth."""
    wl = scenes.small_scene(n=n, seed=3)
    g = oracle.set_dict(wl.sets[0])
    g["opacity_logits"] = np.minimum(g["opacity_logits"], math.log(0.34 / 0.66))
    f = oracle.forward(g, CAM128, margins=oracle.MARGINS_STAGE)
    rgb, T, fl = oracle.render_untiled(f.proj, CAM128, respect_rect=False, margins=oracle.MARGINS_STAGE)
    ok = (f.pixel_flags == 0) & (fl == 0)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(rgb[:, ok], f.image.rgb[:, ok], atol=1e-12)


# ----------------------------------------------------------------------------- backward

def linear_loss(g, cam, w, tile=(16, 16)):
    f = oracle.forward(g, cam, tile)
    return float((f.image.rgb * w).sum()), float(np.abs(f.image.rgb * w).sum())


def fd_check(g, cam, w, keys_idx, tol=1e-6, tile=(16, 16), aabb=None):
    f = oracle.forward(g, cam, tile, margins=oracle.MARGINS_STAGE)
    w = w * (f.pixel_flags == 0)[None]  # no marginal pixel contributes
    g2d, pg = oracle.backward(g, cam, f, w, tile, aabb=aabb)
    worst = 0.0
    for key, idx in keys_idx:
        th = g[key][idx]
        h = 1e-6 * max(1.0, abs(th))
        gp = {k: v.copy() for k, v in g.items()}
        gm = {k: v.copy() for k, v in g.items()}
        gp[key][idx] += h
        gm[key][idx] -= h
        lp, mag = linear_loss(gp, cam, w, tile)
        lm, _ = linear_loss(gm, cam, w, tile)
        fd = (lp - lm) / (2 * h)
        an = getattr(pg, key)[idx]
        scale = np.abs(getattr(pg, key)).max()
        # rounding noise of the difference quotient: a few ulps of the summed loss over 2h
        noise = 8 * np.finfo(float).eps * mag / (2 * h)
        err = max(0.0, abs(fd - an) - noise) / max(abs(an), 1e-3 * scale, 1e-12)
        worst = max(worst, err)
        assert err < tol, (key, idx, fd, an)
    return worst, g2d, pg


def test_backward_matches_finite_differences_all_params_64():
    wl = scenes.small_scene(n=64, seed=4)
    g = oracle.set_dict(wl.sets[0])
    w = np.random.default_rng(1).standard_normal((3, 128, 128))
    keys = []
    for key, shape in [("means", (64, 3)), ("log_scales", (64, 3)), ("quats", (64, 4)),
                       ("opacity_logits", (64,)), ("sh", (64, 16, 3))]:
        keys += [(key, idx) for idx in np.ndindex(*shape)]
    fd_check(g, CAM128, w, keys)


def test_backward_matches_finite_differences_sampled_1k_posed_camera():
    wl = scenes.small_scene()
    g = oracle.set_dict(wl.sets[0])
    vm = scenes.look_at((0.8, -0.6, -0.5), (0.0, 0.0, 4.0), up=(0, -1, 0))
    cam = dict(CAM128, viewmat=vm)
    w = np.random.default_rng(2).standard_normal((3, 128, 128))
    rng = np.random.default_rng(3)
    keys = []
    for key, shape in [("means", (1000, 3)), ("log_scales", (1000, 3)), ("quats", (1000, 4)),
                       ("opacity_logits", (1000,)), ("sh", (1000, 16, 3))]:
        for _ in range(40):
            keys.append((key, tuple(int(rng.integers(0, s)) for s in shape)))
    fd_check(g, cam, w, keys)


def test_sd_statistic_is_scaled_mean2d_gradient_norm():
    wl = scenes.small_scene(n=200)
    g = oracle.set_dict(wl.sets[0])
    f = oracle.forward(g, CAM128)
    w = np.random.default_rng(7).standard_normal((3, 128, 128))
    box = scenes.AABB((-0.5, -0.5, -math.inf), (0.5, 0.5, math.inf))
    g2d, pg = oracle.backward(g, CAM128, f, w, aabb=box)
    inside = (np.abs(g["means"][:, 0] + 0.5 - 0.5) <= 0.5)
    inside = (g["means"][:, 0] >= -0.5) & (g["means"][:, 0] < 0.5) & (g["means"][:, 1] >= -0.5) & (g["means"][:, 1] < 0.5)
    vis = f.proj.radius > 0
    want = np.where(inside & vis, np.hypot(g2d.mean2d[:, 0] * 64, g2d.mean2d[:, 1] * 64), 0.0)
    np.testing.assert_allclose(pg.sd_acc, want, rtol=1e-14, atol=0)
    np.testing.assert_array_equal(pg.sd_cnt, (inside & vis).astype(np.int32))


def test_render_backward_colour_gradient_is_blend_weight():
    """dL/dc_i summed over pixels equals sum_p alpha_i T_i dL/dC_p: with dL/dC = 1 in one
    channel and the image linear in colour, check against FD on the colour directly."""
    wl = scenes.small_scene(n=100)
    g = oracle.set_dict(wl.sets[0])
    f = oracle.forward(g, CAM128)
    w = np.zeros((3, 128, 128))
    w[1] = 1.0
    g2d = oracle.render_bwd(f.proj, f.ids, f.tile_start, CAM128, w)
    # colour enters linearly: perturbing colour i by 1 changes sum(G channel) by sum alpha T
    p = f.proj
    for i in [0, 17, 55]:
        if p.radius[i] == 0:
            continue
        p2 = oracle.Projection(p.mean2d, p.conic, p.color.copy(), p.opacity, p.depth, p.radius, p.rect,
                               p.flags, p.radius_all)
        p2.color[i, 1] += 1.0
        im2 = oracle.render_fwd(p2, f.ids, f.tile_start, CAM128)
        np.testing.assert_allclose(g2d.color[i, 1], (im2.rgb[1] - f.image.rgb[1]).sum(), rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- threshold rules

Y00 = 0.5 / math.sqrt(math.pi)  # the degree-0 real SH constant, 1 / (2 sqrt(pi))
CAM_AXIS = dict(CAM128, cx=64.5, cy=64.5)  # pixel (64, 64) has its centre on the optical axis


def on_axis_stack(logits, dc, z0=2.0, dz=0.5):
    """Gaussians on the optical axis at increasing depths, degree-0 colours dc [n, 3]."""
    n = len(logits)
    sh = np.zeros((n, 16, 3))
    sh[:, 0, :] = dc
    return dict(means=np.stack([np.zeros(n), np.zeros(n), z0 + dz * np.arange(n)], 1),
                log_scales=np.full((n, 3), -4.0), quats=np.tile([1.0, 0, 0, 0], (n, 1)),
                opacity_logits=np.asarray(logits, float), sh=sh)


def test_stop_rule_on_a_stack_closed_form():
    """Twenty Gaussians of opacity 1/2 centred on one pixel centre at increasing depths: each
    has sigma = 0 and alpha = 1/2 there, so T after k of them is 2^-k. The 3DGS stop rule
    (appendix "3DGS Training"; read as: stop before blending a Gaussian when T (1 - alpha) <
    1e-4, that Gaussian excluded) blends exactly 13, since 2^-14 < 1e-4 <= 2^-13: n_contrib = 13,
    T_final = 2^-13, C = sum_{k<13} c_k 2^-(k+1) + T_final bg (the blending equation, Sec. 3.2)."""
    n = 20
    dc = np.linspace(-1.0, 1.0, n)[:, None] * np.array([1.0, 0.5, -0.5])
    g = on_axis_stack(np.zeros(n), dc)
    bg = (0.2, 0.3, 0.4)
    f = oracle.forward(g, CAM_AXIS, bg=bg)
    assert f.image.n_contrib[64, 64] == 13
    assert f.image.T_final[64, 64] == 2.0 ** -13
    col = np.maximum(dc * Y00 + 0.5, 0.0)
    want = (col[:13] * 0.5 ** np.arange(1, 14)[:, None]).sum(0) + 2.0 ** -13 * np.array(bg)
    np.testing.assert_allclose(f.image.rgb[:, 64, 64], want, rtol=1e-12, atol=0)


def test_alpha_clamp_and_one_pixel_adjoint_closed_form():
    """One Gaussian centred on a pixel centre (G = 1 there). Opacity sigmoid(6) = 0.9975: alpha
    is clamped to 0.99 (the 3DGS clamp of appendix "3DGS Training"), so C = 0.99 c + 0.01 bg and
    T = 0.01, and since alpha no longer depends on the opacity past the clamp, that pixel's
    adjoint is dL/do = 0, dL/dc = 0.99 dL/dC. Opacity 1/2: dL/dc = alpha T dL/dC = dL/dC / 2 and
    dL/do = G T (c - bg) . dL/dC (the colour behind the Gaussian is the background)."""
    dc = np.array([[0.8, -0.3, 0.4]])
    col = np.maximum(dc[0] * Y00 + 0.5, 0.0)
    bg = np.array([0.2, 0.3, 0.4])
    w = np.zeros((3, 128, 128))
    w[:, 64, 64] = (0.7, -1.1, 0.5)
    for logit, alpha, clamped in [(6.0, 0.99, True), (0.0, 0.5, False)]:
        g = on_axis_stack([logit], dc)
        f = oracle.forward(g, CAM_AXIS, bg=tuple(bg))
        np.testing.assert_allclose(f.image.rgb[:, 64, 64], alpha * col + (1 - alpha) * bg, rtol=1e-12)
        assert f.image.T_final[64, 64] == 1.0 - alpha
        g2d = oracle.render_bwd(f.proj, f.ids, f.tile_start, CAM_AXIS, w, bg=tuple(bg))
        np.testing.assert_allclose(g2d.color[0], alpha * w[:, 64, 64], rtol=1e-12)
        want_do = 0.0 if clamped else float(np.dot(col - bg, w[:, 64, 64]))
        np.testing.assert_allclose(g2d.opacity[0], want_do, rtol=1e-12, atol=1e-15)


def test_negative_colour_is_clamped_and_passes_no_gradient():
    """The colour is max(0, SH + 1/2) per channel (the 3DGS colour of appendix "3DGS
    Training"): a Gaussian whose degree-0 colour is negative in the green channel composites 0
    there (C = T bg), and the projection adjoint gives that channel's SH coefficients no
    gradient, while the other channels' DC coefficient gets Y00 dL/dc."""
    dc = np.array([[0.8, -3.0, 0.4]])
    g = on_axis_stack([0.0], dc)
    bg = (0.2, 0.3, 0.4)
    f = oracle.forward(g, CAM_AXIS, bg=bg)
    assert f.image.rgb[1, 64, 64] == 0.5 * bg[1]
    g2d = oracle.Grad2D(np.zeros((1, 2)), np.zeros((1, 3)), np.array([[0.3, 0.9, -0.6]]), np.zeros(1))
    pg = oracle.project_bwd(g, CAM_AXIS, g2d)
    np.testing.assert_allclose(pg.sh[0, 0], [Y00 * 0.3, 0.0, Y00 * -0.6], rtol=1e-12)
    assert np.all(pg.sh[0, :, 1] == 0.0)


def test_fov_guard_is_1_3_times_the_half_field_of_view():
    """The culling guard (frustum culling during rasterization, Sec. 3.3; the 3DGS 1.3 x
    half-field-of-view reading): a Gaussian large enough that its footprint reaches the image
    is kept at |x/z| = 1.29 W / (2 fx) and culled at 1.31 W / (2 fx); likewise in y with H, fy
    (a 160 x 96 camera with fx != fy)."""
    cam = dict(CAM128, width=160, height=96, fx=150.0, fy=110.0, cx=80.0, cy=48.0)
    z = 3.0
    hx, hy = 0.5 * 160 / 150.0, 0.5 * 96 / 110.0
    mus = [(1.29 * hx * z, 0, z), (1.31 * hx * z, 0, z), (0, -1.29 * hy * z, z), (0, -1.31 * hy * z, z)]
    g = dict(means=np.array(mus, float), log_scales=np.full((4, 3), -1.2), quats=np.tile([1.0, 0, 0, 0], (4, 1)),
             opacity_logits=np.zeros(4), sh=np.zeros((4, 16, 3)))
    p = oracle.project(g, cam)
    assert list(p.radius > 0) == [True, False, True, False]
    assert np.all(p.radius_all > 0)  # the culled two had footprints that reach the image


def test_principal_point_is_the_image_of_the_optical_axis():
    """A Gaussian on the optical axis projects to the principal point (cx, cy), here with
    cx != cy on a non-square image."""
    cam = dict(CAM128, width=160, height=96, cx=70.25, cy=40.75)
    p = oracle.project(one_gaussian((0.0, 0.0, 3.0), (-3, -3, -3)), cam)
    assert tuple(p.mean2d[0]) == (70.25, 40.75)


def test_sort_breaks_depth_ties_by_index():
    """Equal float32 depths in a tile are ordered by ascending Gaussian index (the tie-break
    reading of the depth sort): 300 Gaussians on five depth planes, against np.lexsort over
    (tile, depth key, index)."""
    rng = np.random.default_rng(8)
    n = 300
    g = dict(means=np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.choice([2.0, 2.5, 3.0, 4.0, 5.0], n)], 1),
             log_scales=rng.uniform(-4, -2, (n, 3)), quats=rng.standard_normal((n, 4)),
             opacity_logits=np.zeros(n), sh=np.zeros((n, 16, 3)))
    p = oracle.project(g, CAM128)
    ids, ts = oracle.bin_sort(p, CAM128)
    tiles, keys, gid = [], [], []
    for i in np.nonzero(p.radius > 0)[0]:
        r = p.rect[i]
        for ty in range(r[1], r[3]):
            for tx in range(r[0], r[2]):
                tiles.append(ty * 8 + tx)
                keys.append(np.float32(p.depth[i]).view(np.uint32))
                gid.append(i)
    tiles, keys, gid = map(np.array, (tiles, keys, gid))
    assert len(np.unique(keys)) == 5  # every list has ties
    order = np.lexsort((gid, keys, tiles))
    np.testing.assert_array_equal(ids, gid[order])


def test_sd_statistic_scales_by_half_width_and_height():
    """The SD statistic (Sec. 3.3) of a view sums ||(dL/du W/2, dL/dv H/2)|| over the views
    where the Gaussian is visible and inside the block: on a 160 x 96 view the two components
    are scaled by 80 and 48."""
    cam = dict(CAM128, width=160, height=96, cx=80.0, cy=48.0)
    wl = scenes.small_scene(n=200)
    g = oracle.set_dict(wl.sets[0])
    f = oracle.forward(g, cam)
    w = np.random.default_rng(9).standard_normal((3, 96, 160))
    g2d, pg = oracle.backward(g, cam, f, w, aabb=scenes.AABB())
    vis = f.proj.radius > 0
    want = np.where(vis, np.hypot(g2d.mean2d[:, 0] * 80, g2d.mean2d[:, 1] * 48), 0.0)
    np.testing.assert_allclose(pg.sd_acc, want, rtol=1e-14, atol=0)


# ----------------------------------------------------------------------------- fast camera selection

def test_depth_composite_on_axis_closed_form():
    """One isotropic Gaussian at depth z on the optical axis: D = z alpha(pixel) exactly
    (a single contributor, T = 1 in front of it), and D / (1 - T_final) = z."""
    s, z = 0.05, 4.0
    g = one_gaussian((0, 0, z), (math.log(s),) * 3, logit=0.4)
    p = oracle.project(g, CAM128)
    ids, ts = oracle.bin_sort(p, CAM128)
    img = oracle.render_depth(p, ids, ts, CAM128)
    var = (128 * s / z) ** 2 + 0.3
    o = 1 / (1 + math.exp(-0.4))
    ys, xs = np.mgrid[0:128, 0:128]
    alpha = np.minimum(0.99, o * np.exp(-((xs + 0.5 - 64) ** 2 + (ys + 0.5 - 64) ** 2) / (2 * var)))
    r = p.radius[0]
    t0, t1 = math.floor((64 - r) / 16), math.ceil((64 + r) / 16)
    seen = (xs // 16 >= t0) & (xs // 16 < t1) & (ys // 16 >= t0) & (ys // 16 < t1) & (alpha >= 1 / 255)
    np.testing.assert_allclose(img.rgb[0], np.where(seen, z * alpha, 0.0), atol=1e-13)
    D = img.rgb[0][seen] / (1 - img.T_final[seen])
    np.testing.assert_allclose(D, z, rtol=1e-12)


def test_depth_of_two_layers_weights_front_and_back():
    """Two concentric isotropic Gaussians at depths z1 < z2 on the axis: at the centre pixel
    D = z1 a1 + z2 a2 (1 - a1)."""
    g = one_gaussian((0, 0, 3.0), (math.log(0.2),) * 3, logit=0.0)
    g2 = one_gaussian((0, 0, 6.0), (math.log(0.4),) * 3, logit=1.0)
    both = {k: np.concatenate([g[k], g2[k]]) for k in g}
    p = oracle.project(both, CAM128)
    ids, ts = oracle.bin_sort(p, CAM128)
    img = oracle.render_depth(p, ids, ts, CAM128)
    rho2 = 0.5 ** 2 * 2  # pixel (64, 64) centre is (64.5, 64.5)
    a1 = 0.5 * math.exp(-rho2 / (2 * ((128 * 0.2 / 3) ** 2 + 0.3)))
    a2 = (1 / (1 + math.exp(-1))) * math.exp(-rho2 / (2 * ((128 * 0.4 / 6) ** 2 + 0.3)))
    assert img.rgb[0][64, 64] == pytest.approx(3.0 * a1 + 6.0 * a2 * (1 - a1), rel=1e-12)


def test_backprojection_inverts_the_pinhole():
    """Back-projected points of a posed camera project back onto their pixel centres at
    camera-space depth D."""
    eye, target = np.array([3.0, -2.0, 5.0]), np.array([0.0, 0.5, 0.0])
    cam = scenes.pinhole(40, 30, 50.0, cx=21.0, cy=14.5, viewmat=scenes.look_at(eye, target)).as_dict()
    rng = np.random.default_rng(3)
    D = rng.uniform(2.0, 9.0, (30, 40))
    T = np.where(rng.uniform(size=(30, 40)) < 0.2, 1.0, rng.uniform(0.0, 0.9, (30, 40)))
    pts, mask = oracle.backproject(D, T, cam)
    assert np.array_equal(mask, T < 1.0)
    V = np.asarray(cam["viewmat"], np.float64)
    pc = pts @ V[:3, :3].T + V[:3, 3]
    ys, xs = np.mgrid[0:30, 0:40]
    np.testing.assert_allclose(pc[..., 2], D, rtol=1e-12)
    np.testing.assert_allclose(cam["fx"] * pc[..., 0] / pc[..., 2] + cam["cx"], xs + 0.5, atol=1e-10)
    np.testing.assert_allclose(cam["fy"] * pc[..., 1] / pc[..., 2] + cam["cy"], ys + 0.5, atol=1e-10)
    # normalised depth divides by the accumulated opacity
    ptsn, _ = oracle.backproject(D, T, cam, normalize=True)
    pcn = ptsn @ V[:3, :3].T + V[:3, 3]
    np.testing.assert_allclose(pcn[..., 2][mask], D[mask] / (1 - T[mask]), rtol=1e-12)


def test_coverage_of_a_wall_split_by_a_block_boundary():
    """A camera facing a wall at depth z along +z (identity pose): the points left of the
    principal point (x < 0 in the world) fall in the block x < 0 -- exactly the pixel columns
    whose centres lie left of cx -- and the ratio V is that fraction."""
    W, H, z = 64, 48, 7.0
    cam = dict(viewmat=np.eye(4), fx=60.0, fy=60.0, cx=27.0, cy=24.0, width=W, height=H, near=0.01, far=1e10)
    D = np.full((H, W), z)
    T = np.zeros((H, W))
    T[:, -5:] = 1.0  # five columns see nothing
    left = scenes.AABB((-math.inf, -math.inf, -math.inf), (0.0, math.inf, math.inf))
    right = scenes.AABB((0.0, -math.inf, -math.inf), (math.inf, math.inf, math.inf))
    near = scenes.AABB((-math.inf, -math.inf, -math.inf), (math.inf, math.inf, z - 1))
    counts, n, _ = oracle.fcs_coverage(D, T, cam, [left, right, near])
    cols_left = int(np.sum(np.arange(W - 5) + 0.5 < 27.0))
    assert n == H * (W - 5)
    assert counts.tolist() == [H * cols_left, H * (W - 5 - cols_left), 0]


def test_coverage_boxes_are_half_open():
    """Block boxes are half-open, lo <= p < hi (the reading of "inside the block" used by the
    partition, Alg. 1): a wall of back-projected points at exactly z = 7 lies in the box
    [7, inf) and not in (-inf, 7)."""
    W, H, z = 32, 24, 7.0
    cam = dict(viewmat=np.eye(4), fx=30.0, fy=30.0, cx=16.0, cy=12.0, width=W, height=H, near=0.01, far=1e10)
    D = np.full((H, W), z)
    T = np.zeros((H, W))
    below = scenes.AABB((-math.inf, -math.inf, -math.inf), (math.inf, math.inf, z))
    above = scenes.AABB((-math.inf, -math.inf, z), (math.inf, math.inf, math.inf))
    counts, n, _ = oracle.fcs_coverage(D, T, cam, [below, above])
    assert counts.tolist() == [0, W * H] and n == W * H


# ----------------------------------------------------------------------------- densification

def dens_set(n=5):
    rng = np.random.default_rng(0)
    return dict(means=rng.standard_normal((n, 3)).astype(np.float32),
                log_scales=np.full((n, 3), -3.0, np.float32), quats=np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
                opacity_logits=np.zeros(n, np.float32), sh=rng.standard_normal((n, 16, 3)).astype(np.float32))


def test_densify_branches_and_order():
    """One Gaussian per branch: pruned (transparent), cloned (large gradient, small), split
    (large gradient, large), kept (small gradient), and a large-gradient Gaussian outside the
    block (no SD views), which is kept."""
    p = dens_set(5)
    p["opacity_logits"][0] = -6.0             # opacity 0.0025 < 0.005
    p["log_scales"][2] = [-1.0, -3.0, -3.0]   # larger than the clone limit
    acc = np.float32([1.0, 0.003, 0.003, 0.0001, 0.0])
    cnt = np.int32([1, 3, 3, 1, 0])
    acc[4] = 5.0                              # no views inside the block: cnt = 0
    normals = np.zeros((5, 2, 3), np.float32)
    out, src = oracle.densify(p, acc, cnt, normals, 2e-4, math.log(0.1), math.log(0.005 / 0.995), 2, math.log(1.6))
    assert src.tolist() == [1, 1, 2, 2, 3, 4]
    np.testing.assert_array_equal(out["means"][0], out["means"][1])  # the clone is an exact copy
    np.testing.assert_allclose(out["log_scales"][2], np.float64([-1.0, -3.0, -3.0]) - math.log(1.6), rtol=1e-15)
    np.testing.assert_allclose(out["means"][2], p["means"][2], rtol=1e-15)  # z = 0: the parent's mean
    np.testing.assert_array_equal(out["sh"][5], p["sh"][4].astype(np.float64))


def test_densify_thresholds_and_sd_views():
    """The densification tests at their thresholds (Sec. 3.3 and the 3DGS density control of
    appendix "3DGS Training", read as: densify when the mean SD gradient reaches the threshold,
    prune when the opacity logit is below the limit, only Gaussians with SD views): a mean
    gradient exactly at the threshold (2^-10 over 4 views = 2^-12) is cloned, a logit exactly at
    the prune limit is kept, and with a zero threshold a Gaussian without SD views (cnt = 0) is
    still only kept."""
    p = dens_set(3)
    p["opacity_logits"][1] = -5.0
    acc = np.float32([2.0 ** -10, 0.0, 0.0])
    cnt = np.int32([4, 1, 0])
    normals = np.zeros((3, 2, 3), np.float32)
    out, src = oracle.densify(p, acc, cnt, normals, 2.0 ** -12, math.log(0.1), -5.0, 2, math.log(1.6))
    assert src.tolist() == [0, 0, 1, 2]
    out, src = oracle.densify(p, acc, cnt, normals, 0.0, math.log(0.1), -6.0, 2, math.log(1.6))
    assert src.tolist() == [0, 0, 1, 1, 2]  # cnt > 0 densifies at threshold 0; cnt = 0 does not


def test_split_child_is_the_rotated_scaled_draw():
    """A 90-degree turn about z with scales (2, 1, 0.5): the draw z = (1, 0, 0) lands at
    mu + (0, 2, 0), z = (0, 0, 1) at mu + (0, 0, 0.5)."""
    p = dens_set(1)
    c, s = math.cos(math.pi / 4), math.sin(math.pi / 4)
    p["quats"][0] = [c, 0, 0, s]
    p["log_scales"][0] = np.log([2.0, 1.0, 0.5])
    normals = np.float32([[[1, 0, 0], [0, 0, 1]]])
    out, src = oracle.densify(p, np.float32([1.0]), np.int32([1]), normals, 2e-4, math.log(0.1), -20.0, 2, math.log(1.6))
    assert src.tolist() == [0, 0]
    np.testing.assert_allclose(out["means"][0] - p["means"][0], [0, 2, 0], atol=1e-6)
    np.testing.assert_allclose(out["means"][1] - p["means"][0], [0, 0, 0.5], atol=1e-6)


def test_split_children_follow_the_gaussian():
    """Children drawn with many standard normals have the parent's covariance R S^2 R^T (the
    split samples from the Gaussian itself)."""
    rng = np.random.default_rng(5)
    m = 200_000
    p = dens_set(1)
    q = rng.standard_normal(4)
    p["quats"][0] = q / np.linalg.norm(q)
    p["log_scales"][0] = np.log([0.3, 0.1, 0.05])
    normals = rng.standard_normal((1, m, 3)).astype(np.float32)
    p1 = {k: np.repeat(v, 1, axis=0) for k, v in p.items()}
    out, _ = oracle.densify(p1, np.float32([1.0]), np.int32([1]), normals, 2e-4, -10.0, -20.0, m, 0.0)
    d = out["means"] - p["means"][0]
    qn = p["quats"][0].astype(np.float64)
    r, x, y, z = qn / np.linalg.norm(qn)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - r * z), 2 * (x * z + r * y)],
                  [2 * (x * y + r * z), 1 - 2 * (x * x + z * z), 2 * (y * z - r * x)],
                  [2 * (x * z - r * y), 2 * (y * z + r * x), 1 - 2 * (x * x + y * y)]])
    Sig = R @ np.diag([0.3, 0.1, 0.05]) ** 2 @ R.T
    np.testing.assert_allclose(np.cov(d.T), Sig, atol=0.01 * 0.09)


# ----------------------------------------------------------------------------- KD partition

def test_kd_partition_bisection_closed_form():
    """Ten cameras, camera k seeing only the point x = k: the median cut (x = 5) leaves 4 / 6
    cameras, the bisection moves right to q = 0.7 (x = 7: 6 / 4), back to q = 0.6 (x = 6:
    5 / 5) and stops there."""
    xs = np.linspace(0.0, 10.0, 1001)
    centers = np.stack([xs, np.linspace(0.0, 1.0, 1001), np.zeros(1001)], 1)
    cams = [np.array([[k + 0.0, 0.5, 0.0]]) for k in range(1, 11)]
    root = scenes.AABB((-math.inf,) * 3, (math.inf,) * 3)
    leaves = oracle.kd_partition(centers, root, 2, cams)
    (lo0, hi0, c0), (lo1, hi1, c1) = leaves
    assert hi0[0] == pytest.approx(6.0) and lo1[0] == pytest.approx(6.0)
    assert c0 == [0, 1, 2, 3, 4] and c1 == [5, 6, 7, 8, 9]


def test_kd_partition_invariants():
    """n_blocks leaves that split the root: every centre in exactly one leaf; the split axis
    follows the longer extent and the cut stays inside the [10%, 90%] percentiles."""
    rng = np.random.default_rng(4)
    centers = np.stack([rng.uniform(-40, 40, 20000), rng.uniform(-10, 10, 20000), np.zeros(20000)], 1)
    cams = [np.stack([rng.normal(cx, 8, 300), rng.normal(cy, 3, 300), np.zeros(300)], 1)
            for cx, cy in zip(rng.uniform(-40, 40, 24), rng.uniform(-10, 10, 24))]
    root = scenes.AABB((-math.inf,) * 3, (math.inf,) * 3)
    leaves = oracle.kd_partition(centers, root, 6, cams)
    assert len(leaves) == 6
    owner = np.zeros(len(centers), int)
    for lo, hi, cs in leaves:
        owner += np.all((centers >= lo) & (centers < hi), axis=1)
        assert set(cs) <= set(range(24))
    assert np.all(owner == 1)
    # two leaves: the cut is along x (80 m against 20 m of extent), near the centres' median
    (lo0, hi0, _), (lo1, hi1, _) = oracle.kd_partition(centers, root, 2, cams)
    assert np.isinf(hi0[1]) and np.isfinite(hi0[0]) and hi0[0] == lo1[0]
    assert np.quantile(centers[:, 0], 0.1) <= hi0[0] <= np.quantile(centers[:, 0], 0.9)


def kd_strip():
    """Centres on a 10 x 1 strip (x in [0, 10], median x = 5) and an unbounded root box."""
    xs = np.linspace(0.0, 10.0, 1001)
    centers = np.stack([xs, np.linspace(0.0, 1.0, 1001), np.zeros(1001)], 1)
    return centers, scenes.AABB((-math.inf,) * 3, (math.inf,) * 3)


def test_kd_partition_keeps_a_camera_at_exactly_tau():
    """A child's camera set keeps a camera whose ratio V reaches tau (Alg. 1, V >= tau): camera
    0 has 1 of its 10 points left of the median cut x = 5 (V = 0.1 = tau), camera 1 has 1 of 10
    right of it; the counts tie at the median, so the cut stays there and both children keep
    both cameras."""
    centers, root = kd_strip()
    cams = [np.array([[2.0, 0.5, 0.0]] + [[8.0, 0.5, 0.0]] * 9), np.array([[2.0, 0.5, 0.0]] * 9 + [[8.0, 0.5, 0.0]])]
    (lo0, hi0, c0), (lo1, hi1, c1) = oracle.kd_partition(centers, root, 2, cams, tau=0.1)
    assert hi0[0] == 5.0 and c0 == [0, 1] and c1 == [0, 1]


def test_kd_partition_splits_the_heaviest_leaf_earliest_first():
    """Alg. 1 splits the leaf with the largest workload (|C(B)|) next, the earliest created
    among equals; one evaluated cut (steps = 1) keeps every cut at the median. One camera left
    of x = 5 and three right of it: the right child (three cameras) is split next, at the
    median of its centres x = 5.00 ... 10.00, 7.5. Two and two: the children tie and the left
    one, created first, is split, at the median of x = 0.00 ... 4.99, 2.495."""
    centers, root = kd_strip()
    pts = lambda xs: [np.array([[x, 0.5, 0.0]]) for x in xs]
    leaves = oracle.kd_partition(centers, root, 3, pts([2.0, 6.0, 8.0, 9.0]), steps=1)
    assert [(lo[0], hi[0]) for lo, hi, _ in leaves] == \
        [(-math.inf, 5.0), (5.0, pytest.approx(7.5)), (pytest.approx(7.5), math.inf)]
    leaves = oracle.kd_partition(centers, root, 3, pts([1.0, 3.0, 7.0, 9.0]), steps=1)
    assert [(lo[0], hi[0]) for lo, hi, _ in leaves] == \
        [(5.0, math.inf), (-math.inf, pytest.approx(2.495)), (pytest.approx(2.495), 5.0)]


# ----------------------------------------------------------------------------- Adam

ADAM_LR = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, opacity_logits=5e-2, sh_dc=2.5e-3, sh_rest=2.5e-3 / 20)


def adam_state(rng, n, scale=1.0):
    shapes = dict(means=(n, 3), log_scales=(n, 3), quats=(n, 4), opacity_logits=(n,), sh=(n, 16, 3))
    return {k: rng.standard_normal(s) * scale for k, s in shapes.items()}


def test_adam_constant_gradient_closed_form():
    """From zero moments under a constant gradient g the bias corrections are exact:
    m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so every step moves p by lr g / (|g| + eps)."""
    rng = np.random.default_rng(0)
    p0, g = adam_state(rng, 5), adam_state(rng, 5, 1e-3)
    p, m, v = p0, {k: np.zeros_like(a) for k, a in p0.items()}, {k: np.zeros_like(a) for k, a in p0.items()}
    for t in range(1, 6):
        p, m, v = oracle.adam(p, g, m, v, t, ADAM_LR, eps=1e-8)
    for k in oracle.ADAM_KEYS:
        rate = np.full(p0[k].shape[1:], ADAM_LR["sh_rest"]) if k == "sh" else ADAM_LR[k]
        if k == "sh":
            rate[0, :] = ADAM_LR["sh_dc"]
        np.testing.assert_allclose(p[k], p0[k] - 5 * rate * g[k] / (np.abs(g[k]) + 1e-8), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(m[k], (1 - 0.9 ** 5) * g[k], rtol=1e-12)
        np.testing.assert_allclose(v[k], (1 - 0.999 ** 5) * g[k] ** 2, rtol=1e-12)


def test_adam_matches_torch_optim():
    """Four steps of random gradients against torch.optim.Adam (library routine) in float64,
    one parameter group per learning rate (the SH split into its degree-0 and other bands)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    n = 7
    p = adam_state(rng, n)
    tp = {k: torch.tensor(a, requires_grad=True) for k, a in p.items() if k != "sh"}
    tp["sh_dc"] = torch.tensor(p["sh"][:, :1, :], requires_grad=True)
    tp["sh_rest"] = torch.tensor(p["sh"][:, 1:, :], requires_grad=True)
    opt = torch.optim.Adam([{"params": [tp[k]], "lr": ADAM_LR[k]} for k in tp], betas=(0.9, 0.999), eps=1e-15)
    m = {k: np.zeros_like(a) for k, a in p.items()}
    v = {k: np.zeros_like(a) for k, a in p.items()}
    for t in range(1, 5):
        g = adam_state(rng, n, 10.0 ** rng.uniform(-6, 0))
        g["means"][0] = 0.0  # a row without gradient this step still moves (momentum)
        for k in tp:
            src = g["sh"][:, :1, :] if k == "sh_dc" else g["sh"][:, 1:, :] if k == "sh_rest" else g[k]
            tp[k].grad = torch.tensor(src)
        opt.step()
        p, m, v = oracle.adam(p, g, m, v, t, ADAM_LR)
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        np.testing.assert_allclose(p[k], tp[k].detach().numpy(), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(p["sh"][:, :1], tp["sh_dc"].detach().numpy(), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(p["sh"][:, 1:], tp["sh_rest"].detach().numpy(), rtol=1e-12, atol=1e-15)
    st = opt.state[tp["quats"]]
    np.testing.assert_allclose(m["quats"], st["exp_avg"].numpy(), rtol=1e-12)
    np.testing.assert_allclose(v["quats"], st["exp_avg_sq"].numpy(), rtol=1e-12)


def test_adam_sparse_rows_leave_the_others_untouched():
    """Sparse variant: rows outside the mask keep parameters and moments bit for bit; rows in
    it get exactly the dense update."""
    rng = np.random.default_rng(2)
    n = 9
    p, g, m = adam_state(rng, n), adam_state(rng, n, 0.1), adam_state(rng, n, 0.01)
    v = {k: np.abs(a) * 0.01 for k, a in adam_state(rng, n).items()}
    rows = rng.uniform(size=n) < 0.5
    rows[0], rows[1] = True, False
    sp, sm, sv = oracle.adam(p, g, m, v, 7, ADAM_LR, rows=rows)
    dp, dm, dv = oracle.adam(p, g, m, v, 7, ADAM_LR)
    for k in oracle.ADAM_KEYS:
        for got, dense, before in ((sp, dp, p), (sm, dm, m), (sv, dv, v)):
            np.testing.assert_array_equal(got[k][~rows], before[k][~rows])
            np.testing.assert_array_equal(got[k][rows], dense[k][rows])
            assert np.all(dense[k][~rows] != before[k][~rows])
