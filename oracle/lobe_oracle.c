/*
 * lobe_oracle.c -- plain, slow FP64 reference of the differentiable tile rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call this
 * file; only tests/, the smoke check and bench.py's CPU-baseline leg use it. It shares
 * no code, header, table or constant with the CUDA library.
 *
 * What it computes (the 3DGS rasterizer the paper builds on; "vanilla 3DGS procedure"
 * of the appendix "3DGS Training", differentiable rasterization of Sec. 2.1, frustum
 * culling of Sec. 3.3, visibility cropping and selective densification of Sec. 3.3, and
 * the alpha-blending equation of Sec. 3.2 with colour in place of depth):
 *
 *   project   : EWA splatting of each 3D Gaussian into a 2D conic, a 3-sigma radius,
 *               a tile rectangle and a view-dependent colour from real SH (degree <= 3).
 *   bin       : (tile, depth) keys for every (Gaussian, tile-in-rect) pair, sorted by
 *               (tile, fp32 depth bits, Gaussian index).
 *   render    : per pixel front-to-back compositing of its tile's list with the
 *               alpha >= 1/255 skip, the 0.99 alpha clamp and the T < 1e-4 stop.
 *   backward  : the textbook reverse-order adjoint of the composite, then the chain
 *               rule back to means, log-scales, quaternions, opacity logits and SH.
 *
 * Every floating-point quantity is double. Inputs that the GPU sees as float32 are
 * passed in already widened, so both sides start from the same values.
 *
 * Readings of points the paper leaves open:
 *   - camera space is OpenCV (x right, y down, +z forward); pixel (i,j) has centre
 *     (i+0.5, j+0.5); u = fx*x/z + cx, v = fy*y/z + cy.
 *   - cull when z < near or z > far, when |x/z| > 1.3*W/(2fx) or |y/z| > 1.3*H/(2fy),
 *     when det(cov2d) <= 0, or when the tile rectangle is empty; crop_mask[g] == 0
 *     (visibility cropping) culls as well.
 *   - cov2d = J W Sigma W^T J^T + 0.3 I ; radius = ceil(3 sqrt(lambda_max)) with
 *     lambda_max = mid + sqrt(max(0.1, mid^2 - det)).
 *   - tile rectangle = [floor((u-r)/tw), ceil((u+r)/tw)) x [floor((v-r)/th), ceil((v+r)/th))
 *     clamped to the tile grid.
 *   - depth = camera-space z evaluated as ((V20*x + V21*y) + V22*z) + V23 in double,
 *     rounded to float32 for the sort key.
 *   - colour = max(0, sum_k sh_k Y_k(normalize(mu - campos)) + 0.5); opacity = sigmoid(logit).
 *   - alpha = min(0.99, o exp(-sigma)); skip sigma < 0 and alpha < 1/255; stop, before
 *     adding, once T (1 - alpha) < 1e-4; C = sum c_i alpha_i T_i + T_final * bg.
 *   - selective-densification statistic: for a Gaussian with radius > 0 whose mean lies
 *     in the block box (lo <= mu < hi per axis), add |(dL/du * W/2, dL/dv * H/2)| and 1.
 *
 * "Marginal" decisions: a decision that float32 arithmetic could take the other way is
 * flagged so that tests can leave it out (per pixel and per Gaussian). The margins are
 * inputs; see orc_margins below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* margins[]: relative margin on alpha/T/clamp decisions, absolute margin (pixels) on
 * rectangle edges, relative margin on 3*sqrt(lambda) near an integer, absolute margin on
 * the colour clamp, absolute margin on sigma near 0, relative margin on the fov guard. */
enum { M_REL = 0, M_PX = 1, M_RAD = 2, M_COL = 3, M_SIG = 4, M_GUARD = 5, M_COUNT = 6 };

/* per-Gaussian flag bits */
enum {
    F_GUARD = 1,   /* fov-guard decision marginal */
    F_RADIUS = 2,  /* ceil(3 sqrt(lambda)) marginal */
    F_RECT = 4,    /* a rectangle edge within M_PX of a tile boundary */
    F_COLOR = 8,   /* colour clamp marginal (gradient mask) */
    F_GUARD_OUT = 16, /* culled by the fov guard (whether or not that decision is marginal) */
};

/* ------------------------------------------------------------------ small helpers */

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

static float to_f32(double x) { return (float)x; }

static uint32_t f32_bits(double x)
{
    float f = (float)x;
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

/* ------------------------------------------------------------------ real spherical harmonics
 *
 * Real SH with the Condon-Shortley phase, ordered (l, m = -l..l), l <= 3:
 *   Y_l^0  = K_l^0 P_l(z)
 *   Y_l^m  = sqrt(2) K_l^m (-1)^m Q_l^m(z) Re((x+iy)^m)      m > 0
 *   Y_l^-m = sqrt(2) K_l^m (-1)^m Q_l^m(z) Im((x+iy)^m)      m > 0
 * with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), Q_l^m = d^m P_l / dz^m and P_l from
 * Rodrigues' formula P_l(z) = 1/(2^l l!) d^l/dz^l (z^2-1)^l. On the unit sphere
 * (1-z^2)^{m/2} cos(m phi) = Re((x+iy)^m), so this equals the spherical-coordinate form
 * (associated Legendre P_l^m = (-1)^m (1-z^2)^{m/2} Q_l^m). Derivatives are taken of this
 * polynomial in (x,y,z); the chain rule through the normalisation removes the radial part.
 */

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= i;
    return f;
}

static double binom(int n, int k) { return factorial(n) / (factorial(k) * factorial(n - k)); }

/* coefficients c[k] of z^k in d^m/dz^m P_l(z) */
static void legendre_deriv_coeffs(int l, int m, double c[8])
{
    double p[16] = {0};
    /* (z^2-1)^l = sum_j binom(l,j) z^{2j} (-1)^{l-j} */
    for (int j = 0; j <= l; ++j) p[2 * j] = binom(l, j) * (((l - j) & 1) ? -1.0 : 1.0);
    /* differentiate l + m times */
    for (int d = 0; d < l + m; ++d)
        for (int k = 0; k < 15; ++k) p[k] = p[k + 1] * (k + 1);
    double s = 1.0 / (pow(2.0, l) * factorial(l));
    for (int k = 0; k < 8; ++k) c[k] = p[k] * s;
}

static double poly_eval(const double c[8], double z, double *dz)
{
    double v = 0.0, d = 0.0;
    for (int k = 7; k >= 0; --k) v = v * z + c[k];
    for (int k = 7; k >= 1; --k) d = d * z + k * c[k];
    if (dz) *dz = d;
    return v;
}

/* (x+iy)^m as (re, im) together with its x,y derivatives */
static void cpow_xy(double x, double y, int m, double *re, double *im,
                    double *dre_dx, double *dre_dy, double *dim_dx, double *dim_dy)
{
    double r = 1.0, i = 0.0, rm1 = 1.0, im1 = 0.0; /* w^m and w^(m-1) */
    for (int k = 0; k < m; ++k) {
        rm1 = r;
        im1 = i;
        double nr = r * x - i * y;
        double ni = r * y + i * x;
        r = nr;
        i = ni;
    }
    *re = r;
    *im = i;
    if (m == 0) {
        *dre_dx = *dre_dy = *dim_dx = *dim_dy = 0.0;
    } else {
        /* d/dx w^m = m w^(m-1);  d/dy w^m = i m w^(m-1) */
        *dre_dx = m * rm1;
        *dim_dx = m * im1;
        *dre_dy = -m * im1;
        *dim_dy = m * rm1;
    }
}

/* Y[16] and dY/d(x,y,z)[16][3] of the polynomial form at (x,y,z). */
void orc_sh_basis(int degree, const double dir[3], double *Y, double *dY)
{
    int k = 0;
    for (int l = 0; l <= degree; ++l) {
        for (int mm = -l; mm <= l; ++mm, ++k) {
            int m = mm < 0 ? -mm : mm;
            double c[8];
            legendre_deriv_coeffs(l, m, c);
            double K = sqrt((2 * l + 1) / (4.0 * ORC_PI) * factorial(l - m) / factorial(l + m));
            double dq;
            double q = poly_eval(c, dir[2], &dq);
            double re, im, drx, dry, dix, diy;
            cpow_xy(dir[0], dir[1], m, &re, &im, &drx, &dry, &dix, &diy);
            double A, dAx, dAy, pre;
            if (mm == 0) {
                A = 1.0; dAx = dAy = 0.0; pre = K;
            } else if (mm > 0) {
                A = re; dAx = drx; dAy = dry; pre = sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);
            } else {
                A = im; dAx = dix; dAy = diy; pre = sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);
            }
            Y[k] = pre * q * A;
            if (dY) {
                dY[3 * k + 0] = pre * q * dAx;
                dY[3 * k + 1] = pre * q * dAy;
                dY[3 * k + 2] = pre * dq * A;
            }
        }
    }
    for (; k < 16; ++k) {
        Y[k] = 0.0;
        if (dY) dY[3 * k] = dY[3 * k + 1] = dY[3 * k + 2] = 0.0;
    }
}

/* ------------------------------------------------------------------ camera */

typedef struct {
    double V[16];
    double fx, fy, cx, cy;
    int W, H;
    double near_plane, far_plane;
    double campos[3];
} cam_t;

/* cam[]: viewmat (16, row-major world->camera), fx, fy, cx, cy, width, height, near, far */
static void load_cam(const double *c, cam_t *k)
{
    memcpy(k->V, c, 16 * sizeof(double));
    k->fx = c[16]; k->fy = c[17]; k->cx = c[18]; k->cy = c[19];
    k->W = (int)c[20]; k->H = (int)c[21];
    k->near_plane = c[22]; k->far_plane = c[23];
    /* camera centre of a rigid transform [R|t]: -R^T t */
    for (int i = 0; i < 3; ++i)
        k->campos[i] = -(k->V[0 + i] * k->V[3] + k->V[4 + i] * k->V[7] + k->V[8 + i] * k->V[11]);
}

/* ------------------------------------------------------------------ 3x3 helpers */

static void quat_to_rot(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR/dq_c for c in {w,x,y,z}: out[c][9] */
static void quat_to_rot_grad(const double q[4], double dR[4][9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], Dw, sizeof Dw);
    memcpy(dR[1], Dx, sizeof Dx);
    memcpy(dR[2], Dy, sizeof Dy);
    memcpy(dR[3], Dz, sizeof Dz);
}

static void mat3_mul(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void mat3_transpose(const double A[9], double T[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * i + j] = A[3 * j + i];
}

/* ------------------------------------------------------------------ projection of one Gaussian */

typedef struct {
    int visible;
    int flags;
    double pc[3];       /* camera-space mean */
    double depth;       /* z as evaluated for the key */
    double mean2d[2];
    double cov2d[3];    /* a, b, c of the dilated 2x2 covariance */
    double conic[3];
    int radius;
    int rect[4];        /* xmin, ymin, xmax, ymax (tiles, max exclusive) */
    double color[3];
    double color_raw[3];
    double opacity;
    double R[9], s[3], qn[3 + 1], qnorm;
    double Sigma[9], Sigma_c[9], J[6];
    double dir[3], dirlen, n[3];
    double Y[16];
} proj_t;

/* Optional per-Gaussian overrides of decisions that float32 arithmetic could take the other
 * way (tests set them to evaluate the other branch; NULL = none). g_vis_flip[g] != 0 inverts
 * the culling decision of Gaussian g in orc_project_bwd; bit ch of g_color_flip[g] inverts
 * the clamp of colour channel ch at 0 in orc_project_bwd. They change no arithmetic. */
static const uint8_t *g_vis_flip = NULL;
static const uint8_t *g_color_flip = NULL;

void orc_set_branch_flips(const uint8_t *vis_flip, const uint8_t *color_flip)
{
    g_vis_flip = vis_flip;
    g_color_flip = color_flip;
}

static int near_integer(double x, double margin)
{
    return fabs(x - floor(x + 0.5)) < margin;
}

static void tile_rect(double u, double v, int r, int tw, int th, int gx, int gy, int rect[4])
{
    rect[0] = (int)clampd(floor((u - r) / tw), 0, gx);
    rect[1] = (int)clampd(floor((v - r) / th), 0, gy);
    rect[2] = (int)clampd(ceil((u + r) / tw), 0, gx);
    rect[3] = (int)clampd(ceil((v + r) / th), 0, gy);
}

static void project_one(const double *mu, const double *ls, const double *q, double logit,
                        const double *sh, int degree, int cropped, const cam_t *k,
                        int tw, int th, const double *mg, int flip_vis, proj_t *P)
{
    memset(P, 0, sizeof *P);
    if (cropped) return;
    const double *V = k->V;
    /* camera-space mean; each component as ((V0*x + V1*y) + V2*z) + V3 */
    for (int i = 0; i < 3; ++i)
        P->pc[i] = ((V[4 * i + 0] * mu[0] + V[4 * i + 1] * mu[1]) + V[4 * i + 2] * mu[2]) + V[4 * i + 3];
    double x = P->pc[0], y = P->pc[1], z = P->pc[2];
    P->depth = z;
    if (!(z >= k->near_plane && z <= k->far_plane)) return;
    double limx = 1.3 * (0.5 * k->W) / k->fx, limy = 1.3 * (0.5 * k->H) / k->fy;
    double txz = x / z, tyz = y / z;
    if (fabs(fabs(txz) - limx) < mg[M_GUARD] * limx || fabs(fabs(tyz) - limy) < mg[M_GUARD] * limy)
        P->flags |= F_GUARD;
    /* the guard decision is applied at the end so that a culled Gaussian still carries
     * the radius and rectangle it would have had (used to flag marginal pixels) */
    int guard_out = fabs(txz) > limx || fabs(tyz) > limy;
    if (guard_out) P->flags |= F_GUARD_OUT;

    /* 3D covariance Sigma = R S S^T R^T */
    P->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) P->qn[i] = q[i] / P->qnorm;
    quat_to_rot(P->qn, P->R);
    for (int i = 0; i < 3; ++i) P->s[i] = exp(ls[i]);
    double M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = P->R[3 * i + j] * P->s[j];
    double Mt[9];
    mat3_transpose(M, Mt);
    mat3_mul(M, Mt, P->Sigma);
    /* camera-frame covariance W Sigma W^T */
    double W[9] = {V[0], V[1], V[2], V[4], V[5], V[6], V[8], V[9], V[10]}, Wt[9], T1[9];
    mat3_transpose(W, Wt);
    mat3_mul(W, P->Sigma, T1);
    mat3_mul(T1, Wt, P->Sigma_c);
    /* perspective Jacobian */
    double *J = P->J;
    J[0] = k->fx / z; J[1] = 0.0;       J[2] = -k->fx * x / (z * z);
    J[3] = 0.0;       J[4] = k->fy / z; J[5] = -k->fy * y / (z * z);
    double JS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int t = 0; t < 3; ++t) s += J[3 * i + t] * P->Sigma_c[3 * t + j];
            JS[3 * i + j] = s;
        }
    double c00 = 0, c01 = 0, c11 = 0;
    for (int t = 0; t < 3; ++t) {
        c00 += JS[t] * J[t];
        c01 += JS[t] * J[3 + t];
        c11 += JS[3 + t] * J[3 + t];
    }
    c00 += 0.3;
    c11 += 0.3;
    P->cov2d[0] = c00; P->cov2d[1] = c01; P->cov2d[2] = c11;
    double det = c00 * c11 - c01 * c01;
    if (!(det > 0.0)) return;
    P->conic[0] = c11 / det;
    P->conic[1] = -c01 / det;
    P->conic[2] = c00 / det;
    double mid = 0.5 * (c00 + c11);
    double lam = mid + sqrt(fmax(0.1, mid * mid - det));
    double r3 = 3.0 * sqrt(lam);
    if (near_integer(r3, mg[M_RAD] * r3 + 1e-12)) P->flags |= F_RADIUS;
    P->radius = (int)ceil(r3);
    P->mean2d[0] = k->fx * x / z + k->cx;
    P->mean2d[1] = k->fy * y / z + k->cy;
    int gx = (k->W + tw - 1) / tw, gy = (k->H + th - 1) / th;
    tile_rect(P->mean2d[0], P->mean2d[1], P->radius, tw, th, gx, gy, P->rect);
    {
        double e[4] = {P->mean2d[0] - P->radius, P->mean2d[0] + P->radius,
                       P->mean2d[1] - P->radius, P->mean2d[1] + P->radius};
        double t[4] = {tw, tw, th, th};
        double gmax[4] = {gx, gx, gy, gy};
        for (int i = 0; i < 4; ++i) {
            double kk = floor(e[i] / t[i] + 0.5);
            if (kk >= 0 && kk <= gmax[i] && fabs(e[i] - kk * t[i]) < mg[M_PX]) P->flags |= F_RECT;
        }
    }
    int culled = guard_out || P->rect[2] <= P->rect[0] || P->rect[3] <= P->rect[1];
    /* a caller may invert a culling decision that float32 could take the other way */
    if (flip_vis) culled = !culled;
    /* view-dependent colour and opacity, also for a culled Gaussian (the other branch of a
     * marginal culling decision needs them) */
    for (int i = 0; i < 3; ++i) P->dir[i] = mu[i] - k->campos[i];
    P->dirlen = sqrt(P->dir[0] * P->dir[0] + P->dir[1] * P->dir[1] + P->dir[2] * P->dir[2]);
    for (int i = 0; i < 3; ++i) P->n[i] = P->dir[i] / P->dirlen;
    orc_sh_basis(degree, P->n, P->Y, NULL);
    int nb = (degree + 1) * (degree + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += sh[3 * b + ch] * P->Y[b];
        P->color_raw[ch] = s + 0.5;
        P->color[ch] = P->color_raw[ch] < 0.0 ? 0.0 : P->color_raw[ch];
        if (fabs(P->color_raw[ch]) < mg[M_COL]) P->flags |= F_COLOR;
    }
    P->opacity = 1.0 / (1.0 + exp(-logit));
    P->visible = !culled;
}

/* ------------------------------------------------------------------ public: project */

int orc_project(int64_t n, const double *means, const double *log_scales, const double *quats,
                const double *logits, const double *sh, int degree, const uint8_t *crop,
                const double *camv, int tw, int th, const double *margins,
                double *mean2d, double *conic, double *color, double *opacity, double *depth,
                int32_t *radius, int32_t *rect, int32_t *flags, int32_t *radius_all, double *color_raw)
{
    cam_t k;
    load_cam(camv, &k);
    for (int64_t g = 0; g < n; ++g) {
        proj_t P;
        project_one(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], sh + 48 * g, degree,
                    crop ? crop[g] == 0 : 0, &k, tw, th, margins, 0, &P);
        mean2d[2 * g] = P.mean2d[0];
        mean2d[2 * g + 1] = P.mean2d[1];
        for (int i = 0; i < 3; ++i) {
            conic[3 * g + i] = P.conic[i];
            color[3 * g + i] = P.color[i];
        }
        opacity[g] = P.opacity;
        depth[g] = P.depth;
        radius[g] = P.visible ? P.radius : 0;
        for (int i = 0; i < 4; ++i) rect[4 * g + i] = P.visible ? P.rect[i] : 0;
        flags[g] = P.flags;
        if (radius_all) radius_all[g] = P.radius;
        if (color_raw)
            for (int i = 0; i < 3; ++i) color_raw[3 * g + i] = P.color_raw[i];
    }
    return 0;
}

/* ------------------------------------------------------------------ sampling window
 * A pixel window [x0,x1) x [y0,y1) that bin/render/render_bwd restrict themselves to, so a
 * timing run can process a bounded sample of a large image with unchanged per-pixel work
 * (pairs of tiles outside the window are not emitted, pixels outside are not touched).
 * Default: no restriction. It changes no arithmetic. */
static int g_win[4] = {0, 0, 1 << 30, 1 << 30};
/* Optionally several windows at once (tiles and pixels inside any of them); g_win is then
 * their bounding box. At most ORC_MAX_WINDOWS. */
#define ORC_MAX_WINDOWS 64
static int g_nwin = 0;
static int g_wins[ORC_MAX_WINDOWS][4];

void orc_set_window(int x0, int y0, int x1, int y1)
{
    g_win[0] = x0; g_win[1] = y0; g_win[2] = x1; g_win[3] = y1;
    g_nwin = 0;
}

int orc_set_windows(int n, const int32_t *rects)
{
    if (n < 1 || n > ORC_MAX_WINDOWS) return -1;
    g_nwin = n;
    g_win[0] = g_win[1] = 1 << 30;
    g_win[2] = g_win[3] = 0;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < 4; ++j) g_wins[i][j] = rects[4 * i + j];
        if (rects[4 * i] < g_win[0]) g_win[0] = rects[4 * i];
        if (rects[4 * i + 1] < g_win[1]) g_win[1] = rects[4 * i + 1];
        if (rects[4 * i + 2] > g_win[2]) g_win[2] = rects[4 * i + 2];
        if (rects[4 * i + 3] > g_win[3]) g_win[3] = rects[4 * i + 3];
    }
    return 0;
}

/* the pixel lies in the sampling window(s) */
static int pixel_in_window(int px, int py)
{
    if (g_nwin == 0) return 1;
    for (int i = 0; i < g_nwin; ++i)
        if (px >= g_wins[i][0] && px < g_wins[i][2] && py >= g_wins[i][1] && py < g_wins[i][3]) return 1;
    return 0;
}

/* Optional per-Gaussian sums of the absolute values of the per-pixel terms that
 * orc_render_bwd adds up ([n][12], the grad2d layout): the scale against which a float32
 * sum of those terms can be resolved. NULL = not collected. Changes no arithmetic. */
static double *g_abs = NULL;

void orc_set_abs_out(double *a12) { g_abs = a12; }

static int tile_in_window(int tx, int ty, int tw, int th)
{
    if (g_nwin == 0)
        return (tx + 1) * tw > g_win[0] && tx * tw < g_win[2] && (ty + 1) * th > g_win[1] && ty * th < g_win[3];
    for (int i = 0; i < g_nwin; ++i)
        if ((tx + 1) * tw > g_wins[i][0] && tx * tw < g_wins[i][2] && (ty + 1) * th > g_wins[i][1] &&
            ty * th < g_wins[i][3])
            return 1;
    return 0;
}

/* ------------------------------------------------------------------ public: bin + sort */

typedef struct {
    uint32_t tile;
    uint32_t dbits;
    int32_t g;
} pair_t;

static int pair_cmp(const void *a, const void *b)
{
    const pair_t *p = a, *q = b;
    if (p->tile != q->tile) return p->tile < q->tile ? -1 : 1;
    if (p->dbits != q->dbits) return p->dbits < q->dbits ? -1 : 1;
    return p->g < q->g ? -1 : (p->g > q->g);
}

/* Returns the number of (Gaussian, tile) pairs. When ids/tile_start are non-NULL they
 * receive the Gaussian index of every pair in (tile, depth, index) order and, for every
 * tile t, the first pair index whose tile is >= t (n_tiles + 1 entries). */
int64_t orc_bin(int64_t n, const double *mean2d, const int32_t *radius, const double *depth,
                int W, int H, int tw, int th, int32_t *ids, int32_t *tile_start)
{
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t total = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (radius[g] <= 0) continue;
        int r[4];
        tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius[g], tw, th, gx, gy, r);
        for (int ty = r[1]; ty < r[3]; ++ty)
            for (int tx = r[0]; tx < r[2]; ++tx) total += tile_in_window(tx, ty, tw, th);
    }
    if (!ids) return total;
    pair_t *pairs = malloc(sizeof(pair_t) * (total ? total : 1));
    int64_t k = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (radius[g] <= 0) continue;
        int r[4];
        tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius[g], tw, th, gx, gy, r);
        for (int ty = r[1]; ty < r[3]; ++ty)
            for (int tx = r[0]; tx < r[2]; ++tx) {
                if (!tile_in_window(tx, ty, tw, th)) continue;
                pairs[k].tile = (uint32_t)(ty * gx + tx);
                pairs[k].dbits = f32_bits(depth[g]);
                pairs[k].g = (int32_t)g;
                ++k;
            }
    }
    qsort(pairs, total, sizeof(pair_t), pair_cmp);
    for (int64_t i = 0; i < total; ++i) ids[i] = pairs[i].g;
    int64_t i = 0;
    for (int t = 0; t <= gx * gy; ++t) {
        while (i < total && pairs[i].tile < (uint32_t)t) ++i;
        tile_start[t] = (int32_t)i;
    }
    free(pairs);
    return total;
}

/* ------------------------------------------------------------------ compositing of one pixel */

typedef struct {
    int32_t g;
    double alpha, T, G, dx, dy, sigma;
    int clamped;
} contrib_t;

/* Walks `list` front to back for pixel (px,py). Writes C[3] (without background), the
 * final T, n_contrib, a marginal flag and (optionally) the contributors. */
static void composite_pixel(int px, int py, const int32_t *list, int64_t len,
                            const double *mean2d, const double *conic, const double *color,
                            const double *opacity, const double *mg,
                            double C[3], double *T_out, int32_t *ncontrib, int *marginal,
                            contrib_t *rec, int64_t *nrec, double *wsum)
{
    double T = 1.0, ws = 0.0;
    C[0] = C[1] = C[2] = 0.0;
    int32_t last = 0;
    int marg = 0;
    int64_t nr = 0;
    double pxc = px + 0.5, pyc = py + 0.5;
    for (int64_t i = 0; i < len; ++i) {
        int32_t g = list[i];
        double dx = mean2d[2 * g] - pxc, dy = mean2d[2 * g + 1] - pyc;
        const double *cn = conic + 3 * g;
        double sigma = 0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) + cn[1] * dx * dy;
        if (fabs(sigma) < mg[M_SIG]) marg = 1;
        if (sigma < 0.0) continue;
        double G = exp(-sigma);
        double araw = opacity[g] * G;
        if (fabs(araw - 0.99) < mg[M_REL] * 0.99) marg = 1;
        int clamped = araw >= 0.99;
        double alpha = clamped ? 0.99 : araw;
        if (fabs(alpha * 255.0 - 1.0) < mg[M_REL]) marg = 1;
        if (alpha < 1.0 / 255.0) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - 1e-4) < mg[M_REL] * 1e-4) marg = 1;
        if (Tn < 1e-4) break;
        double w = alpha * T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += color[3 * g + ch] * w;
        ws += w;
        if (rec) {
            rec[nr].g = g; rec[nr].alpha = alpha; rec[nr].T = T; rec[nr].G = G;
            rec[nr].dx = dx; rec[nr].dy = dy; rec[nr].sigma = sigma; rec[nr].clamped = clamped;
        }
        ++nr;
        T = Tn;
        last = (int32_t)(i + 1);
    }
    *T_out = T;
    *ncontrib = last;
    *marginal = marg;
    if (nrec) *nrec = nr;
    if (wsum) *wsum = ws;
}

/* Flags every pixel of the tiles that a marginal Gaussian might or might not cover.
 * Any rectangle reachable by flipping the marginal decision lies between the rectangle of
 * radius r-1 ("inner") and that of radius r+1 ("outer"); the band outer \ inner is
 * flagged. A Gaussian whose culling decision is marginal flags its whole outer rectangle.
 * radius_all[g] is the radius the projection computed whether or not it culled g. */
int orc_flag_marginal_gaussians(int64_t n, const int32_t *gflags, const double *mean2d,
                                const int32_t *radius, const int32_t *radius_all, int W, int H,
                                int tw, int th, int32_t *pxf)
{
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    for (int64_t g = 0; g < n; ++g) {
        if (!(gflags[g] & (F_GUARD | F_RADIUS | F_RECT))) continue;
        if (radius_all[g] <= 0) continue;
        int outer[4], inner[4] = {0, 0, 0, 0};
        tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius_all[g] + 1, tw, th, gx, gy, outer);
        int whole = (gflags[g] & F_GUARD) || radius[g] <= 0;
        if (!whole && radius_all[g] > 1)
            tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius_all[g] - 1, tw, th, gx, gy, inner);
        for (int ty = outer[1]; ty < outer[3]; ++ty)
            for (int tx = outer[0]; tx < outer[2]; ++tx) {
                if (tx >= inner[0] && tx < inner[2] && ty >= inner[1] && ty < inner[3]) continue;
                for (int y = ty * th; y < (ty + 1) * th && y < H; ++y)
                    for (int x = tx * tw; x < (tx + 1) * tw && x < W; ++x) pxf[(int64_t)y * W + x] = 1;
            }
    }
    return 0;
}

/* ------------------------------------------------------------------ public: render forward */

int orc_render_fwd(int W, int H, int tw, int th, const double *mean2d, const double *conic,
                   const double *color, const double *opacity, const int32_t *ids,
                   const int32_t *tile_start, const double *bg, const double *margins,
                   double *rgb, double *T_final, int32_t *n_contrib, int32_t *pxflags, double *wsum)
{
    int gx = (W + tw - 1) / tw;
    int64_t HW = (int64_t)W * H;
    for (int py = g_win[1]; py < H && py < g_win[3]; ++py)
        for (int px = g_win[0]; px < W && px < g_win[2]; ++px) {
            if (!pixel_in_window(px, py)) continue;
            int t = (py / th) * gx + px / tw;
            double C[3], T, ws;
            int32_t nc;
            int marg;
            composite_pixel(px, py, ids + tile_start[t], tile_start[t + 1] - tile_start[t], mean2d, conic,
                            color, opacity, margins, C, &T, &nc, &marg, NULL, NULL, &ws);
            int64_t p = (int64_t)py * W + px;
            for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + p] = C[ch] + T * bg[ch];
            T_final[p] = T;
            n_contrib[p] = nc;
            if (pxflags) pxflags[p] |= marg;
            if (wsum) wsum[p] = ws;
        }
    return 0;
}

/* ------------------------------------------------------------------ public: untiled renders */

typedef struct {
    uint32_t dbits;
    int32_t g;
} dk_t;

static int dk_cmp(const void *a, const void *b)
{
    const dk_t *p = a, *q = b;
    if (p->dbits != q->dbits) return p->dbits < q->dbits ? -1 : 1;
    return p->g < q->g ? -1 : (p->g > q->g);
}

/* Per pixel: every Gaussian with radius > 0 (and, if respect_rect, whose tile rectangle
 * holds the pixel's tile), sorted by (fp32 depth, index), composited with the same rules.
 * No key duplication, no global sort, no tile ranges. */
int orc_render_untiled(int64_t n, int W, int H, int tw, int th, const double *mean2d,
                       const double *conic, const double *color, const double *opacity,
                       const int32_t *radius, const double *depth, int respect_rect,
                       const double *bg, const double *margins, double *rgb, double *T_final,
                       int32_t *pxflags)
{
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    dk_t *all = malloc(sizeof(dk_t) * (n ? n : 1));
    int32_t *list = malloc(sizeof(int32_t) * (n ? n : 1));
    int64_t m = 0;
    for (int64_t g = 0; g < n; ++g)
        if (radius[g] > 0) {
            all[m].dbits = f32_bits(depth[g]);
            all[m].g = (int32_t)g;
            ++m;
        }
    qsort(all, m, sizeof(dk_t), dk_cmp);
    int64_t HW = (int64_t)W * H;
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int tx = px / tw, ty = py / th;
            int64_t len = 0;
            for (int64_t i = 0; i < m; ++i) {
                int32_t g = all[i].g;
                if (respect_rect) {
                    int r[4];
                    tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius[g], tw, th, gx, gy, r);
                    if (tx < r[0] || tx >= r[2] || ty < r[1] || ty >= r[3]) continue;
                }
                list[len++] = g;
            }
            double C[3], T;
            int32_t nc;
            int marg;
            composite_pixel(px, py, list, len, mean2d, conic, color, opacity, margins, C, &T, &nc,
                            &marg, NULL, NULL, NULL);
            int64_t p = (int64_t)py * W + px;
            for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + p] = C[ch] + T * bg[ch];
            T_final[p] = T;
            if (pxflags) pxflags[p] |= marg;
        }
    free(all);
    free(list);
    return 0;
}

/* ------------------------------------------------------------------ public: render backward
 *
 * Textbook reverse-order adjoint of C = sum_i c_i alpha_i T_i + T_N bg. Walking back from
 * the last contributor with B = colour seen behind Gaussian i (B starts as bg):
 *   dL/dc_i     = alpha_i T_i dL/dC
 *   dL/dalpha_i = T_i (c_i - B) . dL/dC,         B <- alpha_i c_i + (1 - alpha_i) B
 *   alpha = o G, G = exp(-sigma) (unclamped): dL/do = dL/dalpha G, dL/dsigma = -dL/dalpha alpha
 *   sigma = 0.5 (a dx^2 + c dy^2) + b dx dy, dx = u - (px + 0.5), dy = v - (py + 0.5)
 * Gradients accumulate (+=) into per-Gaussian arrays.
 */
int orc_render_bwd(int W, int H, int tw, int th, const double *mean2d, const double *conic,
                   const double *color, const double *opacity, const int32_t *ids,
                   const int32_t *tile_start, const double *bg, const double *dL_drgb,
                   double *d_mean2d, double *d_conic, double *d_color, double *d_opacity)
{
    int gx = (W + tw - 1) / tw;
    int64_t HW = (int64_t)W * H;
    double mg[M_COUNT] = {0, 0, 0, 0, 0, 0};
    int64_t maxlen = 0;
    for (int t = 0; t < gx * ((H + th - 1) / th); ++t)
        if (tile_start[t + 1] - tile_start[t] > maxlen) maxlen = tile_start[t + 1] - tile_start[t];
    contrib_t *rec = malloc(sizeof(contrib_t) * (maxlen ? maxlen : 1));
    for (int py = g_win[1]; py < H && py < g_win[3]; ++py)
        for (int px = g_win[0]; px < W && px < g_win[2]; ++px) {
            if (!pixel_in_window(px, py)) continue;
            int64_t p = (int64_t)py * W + px;
            double gC[3] = {dL_drgb[p], dL_drgb[HW + p], dL_drgb[2 * HW + p]};
            if (gC[0] == 0.0 && gC[1] == 0.0 && gC[2] == 0.0) continue;
            int t = (py / th) * gx + px / tw;
            double C[3], T;
            int32_t nc;
            int marg;
            int64_t nr;
            composite_pixel(px, py, ids + tile_start[t], tile_start[t + 1] - tile_start[t], mean2d,
                            conic, color, opacity, mg, C, &T, &nc, &marg, rec, &nr, NULL);
            double B[3] = {bg[0], bg[1], bg[2]};
            for (int64_t i = nr - 1; i >= 0; --i) {
                const contrib_t *r = rec + i;
                int32_t g = r->g;
                const double *c = color + 3 * g;
                double dalpha = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    d_color[3 * g + ch] += r->alpha * r->T * gC[ch];
                    if (g_abs) g_abs[12 * g + 6 + ch] += fabs(r->alpha * r->T * gC[ch]);
                    dalpha += r->T * (c[ch] - B[ch]) * gC[ch];
                    B[ch] = r->alpha * c[ch] + (1.0 - r->alpha) * B[ch];
                }
                if (r->clamped) continue;
                d_opacity[g] += dalpha * r->G;
                double dsig = -dalpha * r->alpha;
                const double *cn = conic + 3 * g;
                d_conic[3 * g + 0] += dsig * 0.5 * r->dx * r->dx;
                d_conic[3 * g + 1] += dsig * r->dx * r->dy;
                d_conic[3 * g + 2] += dsig * 0.5 * r->dy * r->dy;
                d_mean2d[2 * g + 0] += dsig * (cn[0] * r->dx + cn[1] * r->dy);
                d_mean2d[2 * g + 1] += dsig * (cn[1] * r->dx + cn[2] * r->dy);
                if (g_abs) {
                    double *a = g_abs + 12 * g;
                    a[0] += fabs(dsig * (cn[0] * r->dx + cn[1] * r->dy));
                    a[1] += fabs(dsig * (cn[1] * r->dx + cn[2] * r->dy));
                    a[2] += fabs(dsig * 0.5 * r->dx * r->dx);
                    a[3] += fabs(dsig * r->dx * r->dy);
                    a[4] += fabs(dsig * 0.5 * r->dy * r->dy);
                    a[5] += fabs(dalpha * r->G);
                }
            }
        }
    free(rec);
    return 0;
}

/* ------------------------------------------------------------------ admissible branches
 *
 * A float32 evaluation of the rasterizer may take a decision the other way when the FP64
 * value lies within float32 rounding of its threshold. Either outcome is then a correct
 * result of the method at the precision the GPU computes in. The functions below enumerate,
 * per pixel, every outcome reachable by flipping marginal decisions (the "leaves"), so that a
 * test can accept a float32 result exactly when it matches one of them, instead of leaving
 * such pixels out.
 *
 * Marginal decisions of one (pixel, Gaussian) pair, with the margins of orc_margins:
 *   membership  the Gaussian is in the pixel's tile list only under one outcome of a marginal
 *               projection decision (radius, rectangle edge, fov guard: the "uncertain"
 *               members of orc_bin_ext)
 *   sigma < 0   |sigma| < M_SIG
 *   clamp       |o G - 0.99| < M_REL 0.99 (alpha moves by at most the margin; the gradient
 *               changes form)
 *   alpha skip  |255 alpha - 1| < M_REL
 *   stop        |T (1 - alpha) - 1e-4| < M_REL 1e-4
 * The walk is a depth-first search over the pixel's list in compositing order: at a marginal
 * decision it first follows the FP64 outcome, then the other one. Leaves are numbered in
 * that order, so leaf 0 is the plain FP64 composite, and a second walk over the same inputs
 * numbers them identically. An uncertain member whose sigma or alpha test fails by more than
 * the margin is skipped under both outcomes and is not a branch. */

/* Per Gaussian, the tiles (inside the sampling window) it may belong to: certain members (the
 * FP64 rectangle when no projection decision of the Gaussian is marginal, else the rectangle
 * of radius r - 1 of a visible Gaussian without a marginal guard decision) and uncertain
 * members (the rest of the rectangle of radius r + 1 of a Gaussian with a marginal radius,
 * rectangle or guard decision). unc[k] = 0 certain, 1 uncertain and outside the FP64
 * rectangle, 2 uncertain and inside it. Lists in (tile, fp32 depth, index) order as orc_bin;
 * tile_start as orc_bin. Returns the number of entries; with ids == NULL it only counts. */
/* Whether a marginal decision can change a Gaussian's tile rectangle: a marginal guard
 * decision, or a marginal radius / rectangle edge unless the fov guard culls it anyway. */
static int ext_marginal(int32_t flags, int32_t radius_all)
{
    if (radius_all <= 0) return 0;
    if (flags & F_GUARD) return 1;
    if (flags & F_GUARD_OUT) return 0;
    return (flags & (F_RADIUS | F_RECT)) != 0;
}

static int ext_member(int64_t g, int tx, int ty, const double *mean2d, const int32_t *radius,
                      const int32_t *radius_all, const int32_t *gflags, int tw, int th, int gx, int gy)
{
    /* -1: not a member; 0 certain; 1 uncertain, outside the FP64 rectangle; 2 uncertain, inside */
    int marg = ext_marginal(gflags[g], radius_all[g]);
    int own[4] = {0, 0, 0, 0};
    if (radius[g] > 0) tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius[g], tw, th, gx, gy, own);
    int in_own = tx >= own[0] && tx < own[2] && ty >= own[1] && ty < own[3];
    if (!marg) return in_own ? 0 : -1;
    int outer[4], inner[4] = {0, 0, 0, 0};
    tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius_all[g] + 1, tw, th, gx, gy, outer);
    if (!(tx >= outer[0] && tx < outer[2] && ty >= outer[1] && ty < outer[3])) return -1;
    if (!(gflags[g] & F_GUARD) && radius[g] > 0 && radius_all[g] > 1)
        tile_rect(mean2d[2 * g], mean2d[2 * g + 1], radius_all[g] - 1, tw, th, gx, gy, inner);
    if (tx >= inner[0] && tx < inner[2] && ty >= inner[1] && ty < inner[3]) return 0;
    return in_own ? 2 : 1;
}

int64_t orc_bin_ext(int64_t n, const double *mean2d, const int32_t *radius, const int32_t *radius_all,
                    const int32_t *gflags, const double *depth, int W, int H, int tw, int th,
                    int32_t *ids, uint8_t *unc, int32_t *tile_start)
{
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t total = 0;
    pair_t *pairs = NULL;
    for (int pass = 0; pass < 2; ++pass) {
        int64_t k = 0;
        for (int64_t g = 0; g < n; ++g) {
            int marg = ext_marginal(gflags[g], radius_all[g]);
            if (!marg && radius[g] <= 0) continue;
            int r[4];
            tile_rect(mean2d[2 * g], mean2d[2 * g + 1], marg ? radius_all[g] + 1 : radius[g], tw, th, gx, gy, r);
            for (int ty = r[1]; ty < r[3]; ++ty)
                for (int tx = r[0]; tx < r[2]; ++tx) {
                    if (!tile_in_window(tx, ty, tw, th)) continue;
                    if (ext_member(g, tx, ty, mean2d, radius, radius_all, gflags, tw, th, gx, gy) < 0) continue;
                    if (pass == 1) {
                        pairs[k].tile = (uint32_t)(ty * gx + tx);
                        pairs[k].dbits = f32_bits(depth[g]);
                        pairs[k].g = (int32_t)g;
                    }
                    ++k;
                }
        }
        if (pass == 0) {
            total = k;
            if (!ids) return total;
            pairs = malloc(sizeof(pair_t) * (total ? total : 1));
        }
    }
    qsort(pairs, total, sizeof(pair_t), pair_cmp);
    for (int64_t i = 0; i < total; ++i) {
        int tx = (int)(pairs[i].tile % (uint32_t)gx), ty = (int)(pairs[i].tile / (uint32_t)gx);
        ids[i] = pairs[i].g;
        unc[i] = (uint8_t)ext_member(pairs[i].g, tx, ty, mean2d, radius, radius_all, gflags, tw, th, gx, gy);
    }
    int64_t i = 0;
    for (int t = 0; t <= gx * gy; ++t) {
        while (i < total && pairs[i].tile < (uint32_t)t) ++i;
        tile_start[t] = (int32_t)i;
    }
    free(pairs);
    return total;
}

typedef struct {
    int32_t g;
    int64_t pos;  /* position in the pixel's list */
    double alpha, T, G, dx, dy;
    int clamped;
} brec_t;

typedef struct {
    double T, C[3];
    int32_t last;
    int64_t nrec;
} wstate_t;

typedef struct walk_s walk_t;
struct walk_s {
    double pxc, pyc;
    const int32_t *list;
    const uint8_t *unc;  /* NULL: every member certain */
    int64_t len;
    const double *mean2d, *conic, *color, *opacity, *mg;
    int max_leaves, nleaves, overflow;
    brec_t *rec;
    void (*leaf)(walk_t *w, int index, const wstate_t *S);
    void *user;
};

/* one pair's FP64 quantities */
typedef struct {
    int64_t i;
    int32_t g;
    double dx, dy, sigma, G, araw;
} pairq_t;

static void walk(walk_t *w, int64_t i, wstate_t S);

static void emit_leaf(walk_t *w, const wstate_t *S)
{
    if (w->overflow) return;
    if (w->nleaves >= w->max_leaves) {
        w->overflow = 1;
        return;
    }
    w->leaf(w, w->nleaves, S);
    w->nleaves++;
}

/* the stop test and, unless the walk stops, the pair's contribution. A stop leaves the state
 * as it was before the pair, whatever alpha the pair had: *stopped (nullable) records that
 * this pair's stop leaf exists, so that its other outcomes do not repeat it. */
static void pair_stop(walk_t *w, const pairq_t *q, wstate_t S, double alpha, int clamped, int *stopped)
{
    double Tn = S.T * (1.0 - alpha);
    int stop = Tn < 1e-4, marg = fabs(Tn - 1e-4) < w->mg[M_REL] * 1e-4;
    for (int b = 0; b < 1 + marg; ++b) {
        int st = b == 0 ? stop : !stop;
        if (st) {
            if (stopped && *stopped) continue;
            if (stopped) *stopped = 1;
            emit_leaf(w, &S);
            continue;
        }
        wstate_t N = S;
        double wgt = alpha * S.T;
        for (int ch = 0; ch < 3; ++ch) N.C[ch] += w->color[3 * q->g + ch] * wgt;
        brec_t *r = w->rec + S.nrec;
        r->g = q->g; r->pos = q->i; r->alpha = alpha; r->T = S.T; r->G = q->G;
        r->dx = q->dx; r->dy = q->dy; r->clamped = clamped;
        N.nrec = S.nrec + 1;
        N.T = Tn;
        N.last = (int32_t)(q->i + 1);
        walk(w, q->i + 1, N);
    }
}

/* The distinct outcomes of one pair with a marginal decision: "skipped" (not a member, sigma
 * < 0 or alpha < 1/255: all leave the state as it is) and "used with the clamp on / off".
 * The FP64 outcome comes first; only outcomes some assignment of the marginal decisions
 * reaches are followed. u is the pair's membership flag (0 certain, 1 / 2 uncertain with
 * the FP64 rectangle excluding / including it). */
static void pair_branch(walk_t *w, const pairq_t *q, int u, wstate_t S)
{
    const double *mg = w->mg;
    int mem_fp = u != 1, mem_m = u != 0;
    int sig_fp = !(q->sigma < 0.0), sig_m = fabs(q->sigma) < mg[M_SIG];  /* the sigma test passes */
    int cl_fp = q->araw >= 0.99, cl_m = fabs(q->araw - 0.99) < mg[M_REL] * 0.99;
    double a_of[2];
    int pass_fp[2], pass_m[2];
    for (int c = 0; c < 2; ++c) {
        a_of[c] = c ? 0.99 : q->araw;
        pass_fp[c] = !(a_of[c] < 1.0 / 255.0);
        pass_m[c] = fabs(a_of[c] * 255.0 - 1.0) < mg[M_REL];
    }
    int mem_in = mem_fp || mem_m, mem_out = !mem_fp || mem_m;
    int sig_pass = sig_fp || sig_m, sig_fail = !sig_fp || sig_m;
    int use_ok[2], skip_ok = mem_out || (mem_in && sig_fail);
    for (int c = 0; c < 2; ++c) {
        int clamp_ok = c == cl_fp || cl_m;
        use_ok[c] = mem_in && sig_pass && clamp_ok && (pass_fp[c] || pass_m[c]);
        if (mem_in && sig_pass && clamp_ok && (!pass_fp[c] || pass_m[c])) skip_ok = 1;
    }
    int fp_used = mem_fp && sig_fp && pass_fp[cl_fp];
    /* outcome codes: 0 skipped, 1 used unclamped, 2 used clamped; FP64 first */
    int order[3], no = 0;
    order[no++] = fp_used ? 1 + cl_fp : 0;
    if (order[0] != 0 && skip_ok) order[no++] = 0;
    for (int c = 0; c < 2; ++c)
        if (use_ok[c] && order[0] != 1 + c) order[no++] = 1 + c;
    int stopped = 0;
    for (int k = 0; k < no; ++k) {
        if (order[k] == 0)
            walk(w, q->i + 1, S);
        else
            pair_stop(w, q, S, a_of[order[k] - 1], order[k] - 1, &stopped);
    }
}

static void walk(walk_t *w, int64_t i, wstate_t S)
{
    const double *mg = w->mg;
    for (; i < w->len; ++i) {
        if (w->overflow) return;
        pairq_t q;
        q.i = i;
        q.g = w->list[i];
        q.dx = w->mean2d[2 * q.g] - w->pxc;
        q.dy = w->mean2d[2 * q.g + 1] - w->pyc;
        const double *cn = w->conic + 3 * q.g;
        q.sigma = 0.5 * (cn[0] * q.dx * q.dx + cn[2] * q.dy * q.dy) + cn[1] * q.dx * q.dy;
        q.G = exp(-q.sigma);
        q.araw = w->opacity[q.g] * q.G;
        int m_sig = fabs(q.sigma) < mg[M_SIG];
        int m_clamp = fabs(q.araw - 0.99) < mg[M_REL] * 0.99;
        double alpha = q.araw >= 0.99 ? 0.99 : q.araw;
        int m_a = fabs(alpha * 255.0 - 1.0) < mg[M_REL];
        int u = w->unc ? w->unc[i] : 0;
        if (u || m_sig || m_clamp || m_a) {
            pair_branch(w, &q, u, S);
            return;
        }
        /* no marginal decision: the plain step */
        if (q.sigma < 0.0 || alpha < 1.0 / 255.0) continue;
        double Tn = S.T * (1.0 - alpha);
        if (fabs(Tn - 1e-4) < mg[M_REL] * 1e-4) {
            pair_stop(w, &q, S, alpha, q.araw >= 0.99, NULL);
            return;
        }
        if (Tn < 1e-4) {
            emit_leaf(w, &S);
            return;
        }
        double wgt = alpha * S.T;
        for (int ch = 0; ch < 3; ++ch) S.C[ch] += w->color[3 * q.g + ch] * wgt;
        brec_t *r = w->rec + S.nrec;
        r->g = q.g; r->pos = i; r->alpha = alpha; r->T = S.T; r->G = q.G;
        r->dx = q.dx; r->dy = q.dy; r->clamped = q.araw >= 0.99;
        S.nrec++;
        S.T = Tn;
        S.last = (int32_t)(i + 1);
    }
    emit_leaf(w, &S);
}

static void walk_pixel(walk_t *w, int px, int py, const int32_t *list, const uint8_t *unc, int64_t len)
{
    w->pxc = px + 0.5;
    w->pyc = py + 0.5;
    w->list = list;
    w->unc = unc;
    w->len = len;
    w->nleaves = 0;
    w->overflow = 0;
    wstate_t S;
    S.T = 1.0;
    S.C[0] = S.C[1] = S.C[2] = 0.0;
    S.last = 0;
    S.nrec = 0;
    walk(w, 0, S);
}

/* forward leaves of a window */
typedef struct {
    int L;
    double *C, *T;
    int32_t *nc;
    const double *bg;
    int64_t p;  /* window pixel index */
} fleaf_t;

static void fwd_leaf(walk_t *w, int index, const wstate_t *S)
{
    fleaf_t *f = w->user;
    int64_t o = f->p * f->L + index;
    for (int ch = 0; ch < 3; ++ch) f->C[3 * o + ch] = S->C[ch] + S->T * f->bg[ch];
    f->T[o] = S->T;
    f->nc[o] = S->last;
}

static int64_t max_tile_len(const int32_t *tile_start, int n_tiles)
{
    int64_t m = 0;
    for (int t = 0; t < n_tiles; ++t)
        if (tile_start[t + 1] - tile_start[t] > m) m = tile_start[t + 1] - tile_start[t];
    return m;
}

/* Every leaf of every pixel of the window [x0,x1) x [y0,y1) (clipped to the image). Window
 * pixel p = (y - y0) * (x1 - x0) + (x - x0) gets nleaf[p] leaves (0 when there are more than
 * max_leaves: the pixel cannot be checked) with colour (background included) C[p][l][3],
 * T_final T[p][l] and n_contrib nc[p][l]. unc may be NULL (all members certain). */
int orc_render_leaves(int W, int H, int tw, int th, const double *mean2d, const double *conic,
                      const double *color, const double *opacity, const int32_t *ids, const uint8_t *unc,
                      const int32_t *tile_start, const double *bg, const double *margins, int x0, int y0,
                      int x1, int y1, int max_leaves, int32_t *nleaf, double *C, double *T, int32_t *nc)
{
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t maxlen = max_tile_len(tile_start, gx * gy);
    walk_t w;
    memset(&w, 0, sizeof w);
    w.mean2d = mean2d; w.conic = conic; w.color = color; w.opacity = opacity; w.mg = margins;
    w.max_leaves = max_leaves;
    w.rec = malloc(sizeof(brec_t) * (maxlen ? maxlen : 1));
    w.leaf = fwd_leaf;
    fleaf_t f = {max_leaves, C, T, nc, bg, 0};
    w.user = &f;
    int ww = x1 - x0;
    for (int py = y0; py < y1 && py < H; ++py)
        for (int px = x0; px < x1 && px < W; ++px) {
            int t = (py / th) * gx + px / tw;
            f.p = (int64_t)(py - y0) * ww + (px - x0);
            walk_pixel(&w, px, py, ids + tile_start[t], unc ? unc + tile_start[t] : NULL,
                       tile_start[t + 1] - tile_start[t]);
            nleaf[f.p] = w.overflow ? 0 : w.nleaves;
        }
    free(w.rec);
    return 0;
}

/* Backward envelope: the textbook reverse-order adjoint (as orc_render_bwd) of every leaf
 * that admissible[p] (bit l = leaf l) lists, per window pixel. Per Gaussian and each of the
 * 12 grad2d components (u, v, conic a, b, c, opacity, r, g, b, 0, 0, 0) lo/hi receive the
 * sum over pixels of the smallest / largest contribution among that pixel's admissible
 * leaves (a Gaussian absent from a leaf contributes 0 there), and absmax the sum over
 * pixels of the largest, over its admissible leaves, absolute per-pixel term: every value a
 * consistent choice of one admissible leaf per pixel can produce lies in [lo, hi]. */
typedef struct {
    const uint64_t *adm;
    int64_t p;
    const double *gC;  /* dL/dC of the pixel */
    const double *bg, *conic, *color;
    /* per list position: current leaf's terms, running min/max/absmax, last leaf seen */
    double *cur, *mn, *mx, *ab;
    int32_t *seen;     /* leaf count (1-based) at the last update of the position, 0 = never */
    int64_t *touched;
    int64_t ntouched;
    int32_t *gid;
    int nadm;          /* admissible leaves folded so far for this pixel */
} bleaf_t;

static void bwd_leaf(walk_t *w, int index, const wstate_t *S)
{
    bleaf_t *b = w->user;
    if (index >= 64 || !((b->adm[b->p] >> index) & 1)) return;
    const double *gC = b->gC;
    double B[3] = {b->bg[0], b->bg[1], b->bg[2]};
    int k = ++b->nadm;
    for (int64_t r = S->nrec - 1; r >= 0; --r) {
        const brec_t *e = w->rec + r;
        int32_t g = e->g;
        const double *c = b->color + 3 * g;
        double t[12] = {0};
        double dalpha = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            t[6 + ch] = e->alpha * e->T * gC[ch];
            dalpha += e->T * (c[ch] - B[ch]) * gC[ch];
            B[ch] = e->alpha * c[ch] + (1.0 - e->alpha) * B[ch];
        }
        if (!e->clamped) {
            const double *cn = b->conic + 3 * g;
            double dsig = -dalpha * e->alpha;
            t[5] = dalpha * e->G;
            t[2] = dsig * 0.5 * e->dx * e->dx;
            t[3] = dsig * e->dx * e->dy;
            t[4] = dsig * 0.5 * e->dy * e->dy;
            t[0] = dsig * (cn[0] * e->dx + cn[1] * e->dy);
            t[1] = dsig * (cn[1] * e->dx + cn[2] * e->dy);
        }
        int64_t pos = e->pos;
        double *cur = b->cur + 12 * pos;
        for (int j = 0; j < 12; ++j) cur[j] = t[j];
        if (b->seen[pos] == 0) {
            /* first time in this pixel: earlier admissible leaves had it absent (0) */
            b->touched[b->ntouched++] = pos;
            b->gid[pos] = g;
            for (int j = 0; j < 12; ++j) {
                b->mn[12 * pos + j] = k > 1 ? fmin(0.0, t[j]) : t[j];
                b->mx[12 * pos + j] = k > 1 ? fmax(0.0, t[j]) : t[j];
                b->ab[12 * pos + j] = fabs(t[j]);
            }
        } else {
            for (int j = 0; j < 12; ++j) {
                b->mn[12 * pos + j] = fmin(b->mn[12 * pos + j], t[j]);
                b->mx[12 * pos + j] = fmax(b->mx[12 * pos + j], t[j]);
                b->ab[12 * pos + j] = fmax(b->ab[12 * pos + j], fabs(t[j]));
            }
        }
        b->seen[pos] = k;
    }
    /* positions of earlier leaves absent from this one contribute 0 here */
    for (int64_t m = 0; m < b->ntouched; ++m) {
        int64_t pos = b->touched[m];
        if (b->seen[pos] == k) continue;
        for (int j = 0; j < 12; ++j) {
            b->mn[12 * pos + j] = fmin(b->mn[12 * pos + j], 0.0);
            b->mx[12 * pos + j] = fmax(b->mx[12 * pos + j], 0.0);
        }
        b->seen[pos] = k;
    }
}

int orc_render_bwd_envelope(int W, int H, int tw, int th, const double *mean2d, const double *conic,
                            const double *color, const double *opacity, const int32_t *ids,
                            const uint8_t *unc, const int32_t *tile_start, const double *bg,
                            const double *margins, int x0, int y0, int x1, int y1, int max_leaves,
                            const uint64_t *admissible, const double *dL_drgb, double *lo, double *hi,
                            double *absmax)
{
    int gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int64_t HW = (int64_t)W * H;
    int64_t maxlen = max_tile_len(tile_start, gx * gy);
    int64_t m1 = maxlen ? maxlen : 1;
    walk_t w;
    memset(&w, 0, sizeof w);
    w.mean2d = mean2d; w.conic = conic; w.color = color; w.opacity = opacity; w.mg = margins;
    w.max_leaves = max_leaves;
    w.rec = malloc(sizeof(brec_t) * m1);
    w.leaf = bwd_leaf;
    bleaf_t b;
    memset(&b, 0, sizeof b);
    b.adm = admissible; b.bg = bg; b.conic = conic; b.color = color;
    b.cur = malloc(sizeof(double) * 12 * m1);
    b.mn = malloc(sizeof(double) * 12 * m1);
    b.mx = malloc(sizeof(double) * 12 * m1);
    b.ab = malloc(sizeof(double) * 12 * m1);
    b.seen = calloc((size_t)m1, sizeof(int32_t));
    b.touched = malloc(sizeof(int64_t) * m1);
    b.gid = malloc(sizeof(int32_t) * m1);
    w.user = &b;
    int ww = x1 - x0;
    for (int py = y0; py < y1 && py < H; ++py)
        for (int px = x0; px < x1 && px < W; ++px) {
            int64_t p = (int64_t)py * W + px;
            double gC[3] = {dL_drgb[p], dL_drgb[HW + p], dL_drgb[2 * HW + p]};
            b.p = (int64_t)(py - y0) * ww + (px - x0);
            if (admissible[b.p] == 0) continue;
            if (gC[0] == 0.0 && gC[1] == 0.0 && gC[2] == 0.0) continue;
            int t = (py / th) * gx + px / tw;
            b.gC = gC;
            b.nadm = 0;
            b.ntouched = 0;
            walk_pixel(&w, px, py, ids + tile_start[t], unc ? unc + tile_start[t] : NULL,
                       tile_start[t + 1] - tile_start[t]);
            for (int64_t m = 0; m < b.ntouched; ++m) {
                int64_t pos = b.touched[m];
                int32_t g = b.gid[pos];
                for (int j = 0; j < 12; ++j) {
                    lo[12 * g + j] += b.mn[12 * pos + j];
                    hi[12 * g + j] += b.mx[12 * pos + j];
                    absmax[12 * g + j] += b.ab[12 * pos + j];
                }
                b.seen[pos] = 0;
            }
        }
    free(w.rec);
    free(b.cur); free(b.mn); free(b.mx); free(b.ab); free(b.seen); free(b.touched); free(b.gid);
    return 0;
}

/* ------------------------------------------------------------------ public: projection backward
 *
 * Chain rule from dL/d(mean2d, conic, colour, opacity) of one view to the raw parameters.
 * Adds into g_* (+=). sd_acc/sd_cnt receive the selective-densification statistic.
 */
int orc_project_bwd(int64_t n, const double *means, const double *log_scales, const double *quats,
                    const double *logits, const double *sh, int degree, const uint8_t *crop,
                    const double *camv, int tw, int th, const double *aabb,
                    const double *d_mean2d, const double *d_conic, const double *d_color,
                    const double *d_opacity, double *g_means, double *g_log_scales,
                    double *g_quats, double *g_logits, double *g_sh, double *sd_acc, int32_t *sd_cnt)
{
    cam_t k;
    load_cam(camv, &k);
    double mg[M_COUNT] = {0, 0, 0, 0, 0, 0};
    const double *V = k.V;
    double W[9] = {V[0], V[1], V[2], V[4], V[5], V[6], V[8], V[9], V[10]};
    for (int64_t g = 0; g < n; ++g) {
        proj_t P;
        const double *mu = means + 3 * g;
        project_one(mu, log_scales + 3 * g, quats + 4 * g, logits[g], sh + 48 * g, degree,
                    crop ? crop[g] == 0 : 0, &k, tw, th, mg, g_vis_flip ? g_vis_flip[g] : 0, &P);
        if (!P.visible) continue;
        double gmu[3] = {0, 0, 0};
        /* opacity */
        g_logits[g] += d_opacity[g] * P.opacity * (1.0 - P.opacity);
        /* colour -> SH and view direction */
        int nb = (degree + 1) * (degree + 1);
        double Y[16], dY[48];
        orc_sh_basis(degree, P.n, Y, dY);
        double dn[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            int clamped = P.color_raw[ch] < 0.0;
            if (g_color_flip && ((g_color_flip[g] >> ch) & 1)) clamped = !clamped;
            if (clamped) continue;
            double dc = d_color[3 * g + ch];
            for (int b = 0; b < nb; ++b) {
                g_sh[48 * g + 3 * b + ch] += Y[b] * dc;
                for (int i = 0; i < 3; ++i) dn[i] += sh[48 * g + 3 * b + ch] * dY[3 * b + i] * dc;
            }
        }
        /* n = dir/|dir|: dn/ddir = (I - n n^T)/|dir| */
        double ndn = P.n[0] * dn[0] + P.n[1] * dn[1] + P.n[2] * dn[2];
        for (int i = 0; i < 3; ++i) gmu[i] += (dn[i] - P.n[i] * ndn) / P.dirlen;

        /* conic = inverse(cov2d): dL/dcov2d = -C Gs C with Gs = [[da, db/2],[db/2, dc]] */
        double C2[4] = {P.conic[0], P.conic[1], P.conic[1], P.conic[2]};
        double Gs[4] = {d_conic[3 * g], 0.5 * d_conic[3 * g + 1], 0.5 * d_conic[3 * g + 1], d_conic[3 * g + 2]};
        double CG[4], H2[4];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) CG[2 * i + j] = C2[2 * i] * Gs[j] + C2[2 * i + 1] * Gs[2 + j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) H2[2 * i + j] = -(CG[2 * i] * C2[j] + CG[2 * i + 1] * C2[2 + j]);
        /* cov2d = J Sigma_c J^T + 0.3 I:  dL/dSigma_c = J^T H J,  dL/dJ = 2 H J Sigma_c */
        const double *J = P.J;
        double dSc[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0;
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) s += J[3 * i + a] * H2[2 * i + j] * J[3 * j + b];
                dSc[3 * a + b] = s;
            }
        double dJ[6];
        for (int i = 0; i < 2; ++i)
            for (int b = 0; b < 3; ++b) {
                double s = 0;
                for (int j = 0; j < 2; ++j)
                    for (int a = 0; a < 3; ++a) s += H2[2 * i + j] * J[3 * j + a] * P.Sigma_c[3 * a + b];
                dJ[3 * i + b] = 2.0 * s;
            }
        /* J and (u,v) as functions of the camera-space mean */
        double x = P.pc[0], y = P.pc[1], z = P.pc[2];
        double fx = k.fx, fy = k.fy;
        double dpc[3] = {0, 0, 0};
        double du = d_mean2d[2 * g], dv = d_mean2d[2 * g + 1];
        dpc[0] += du * fx / z;
        dpc[1] += dv * fy / z;
        dpc[2] += -du * fx * x / (z * z) - dv * fy * y / (z * z);
        /* J00 = fx/z, J02 = -fx x/z^2, J11 = fy/z, J12 = -fy y/z^2 */
        dpc[0] += dJ[2] * (-fx / (z * z));
        dpc[1] += dJ[5] * (-fy / (z * z));
        dpc[2] += dJ[0] * (-fx / (z * z)) + dJ[2] * (2.0 * fx * x / (z * z * z)) +
                  dJ[4] * (-fy / (z * z)) + dJ[5] * (2.0 * fy * y / (z * z * z));
        /* pc = W mu + t */
        for (int i = 0; i < 3; ++i) gmu[i] += W[0 + i] * dpc[0] + W[3 + i] * dpc[1] + W[6 + i] * dpc[2];
        /* Sigma_c = W Sigma W^T -> dL/dSigma = W^T dSc W */
        double Wt[9], T1[9], dS[9];
        mat3_transpose(W, Wt);
        mat3_mul(Wt, dSc, T1);
        mat3_mul(T1, W, dS);
        /* Sigma = M M^T, M = R diag(s): dL/dM = (dS + dS^T) M */
        double M[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[3 * i + j] = P.R[3 * i + j] * P.s[j];
        double dSsym[9], dM[9];
        for (int i = 0; i < 9; ++i) dSsym[i] = dS[i] + dS[3 * (i % 3) + i / 3];
        mat3_mul(dSsym, M, dM);
        double dR[9];
        for (int j = 0; j < 3; ++j) {
            double ds = 0;
            for (int i = 0; i < 3; ++i) {
                ds += dM[3 * i + j] * P.R[3 * i + j];
                dR[3 * i + j] = dM[3 * i + j] * P.s[j];
            }
            g_log_scales[3 * g + j] += ds * P.s[j];
        }
        double dRq[4][9];
        quat_to_rot_grad(P.qn, dRq);
        double dqn[4];
        for (int c = 0; c < 4; ++c) {
            double s = 0;
            for (int i = 0; i < 9; ++i) s += dR[i] * dRq[c][i];
            dqn[c] = s;
        }
        double qd = 0;
        for (int c = 0; c < 4; ++c) qd += P.qn[c] * dqn[c];
        for (int c = 0; c < 4; ++c) g_quats[4 * g + c] += (dqn[c] - P.qn[c] * qd) / P.qnorm;
        for (int i = 0; i < 3; ++i) g_means[3 * g + i] += gmu[i];
        /* selective densification statistic */
        if (aabb && sd_acc) {
            int inside = 1;
            for (int i = 0; i < 3; ++i)
                if (!(mu[i] >= aabb[i] && mu[i] < aabb[3 + i])) inside = 0;
            if (inside) {
                double a = du * 0.5 * k.W, b = dv * 0.5 * k.H;
                sd_acc[g] += sqrt(a * a + b * b);
                sd_cnt[g] += 1;
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ public: visibility crop
 * Sec. 3.3: keep a Gaussian if it is visible (radius > 0 under the culling rules above)
 * from at least one of the block's cameras. mask[g] |= visible. */
int orc_visibility_crop(int64_t n, const double *means, const double *log_scales, const double *quats,
                        const double *logits, const double *sh, int degree, const double *camv,
                        int tw, int th, uint8_t *mask)
{
    cam_t k;
    load_cam(camv, &k);
    double mg[M_COUNT] = {0, 0, 0, 0, 0, 0};
    for (int64_t g = 0; g < n; ++g) {
        proj_t P;
        project_one(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], sh + 48 * g, degree, 0,
                    &k, tw, th, mg, 0, &P);
        if (P.visible) mask[g] = 1;
    }
    return 0;
}

/* float32 rounding helper exported for tests that need the key the GPU sees */
uint32_t orc_depth_key(double z) { return f32_bits(z); }
float orc_round_f32(double x) { return to_f32(x); }
