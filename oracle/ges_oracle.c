/*
 * FP64 CPU oracle for the GES (generalized-exponential splatting) rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. The product path never calls it,
 * and it shares no code, header or constant table with the CUDA library.
 *
 * It computes, per pixel and by brute force over every visible splat in depth
 * order (no tiles, no binning), what the rasterizer must produce:
 *
 *   S1  Sigma = R S' S'^T R^T, S' = phi(beta) * exp(l)           Eq. 4, Eq. 6-7
 *   S2  Sigma' = J W Sigma W^T J^T (+ low-pass h I), conic       EWA projection (Sec. 3.2)
 *   S3  support of the falloff exp(-1/2 Q^(beta/2))               Eq. 3
 *   S4  colour from real spherical harmonics; normal = axis of the smallest
 *       scale, facing the camera                                 Sec. 3.3 (n_g*)
 *   S6  front-to-back alpha compositing of colour, depth, alpha
 *       and normal                                               Eq. 5, discretised
 *   S7  the analytic gradient of S6, and S8 its chain rule back
 *       to the 3-D parameters
 *
 * Readings where the paper is silent (shared with the CUDA side only through
 * this written convention, never through code):
 *   - phi(beta) centred form 2 / (1 + exp(-rho (beta - 2))), mode 1; mode 0 is
 *     phi = 1; mode 2 is the expression as printed in Eq. 7.
 *   - phi multiplies all three scales.
 *   - the falloff is the exact exp(-1/2 Q^(beta/2)) with peak = opacity.
 *   - alpha = min(alpha_max, o G); splats with alpha < alpha_min are skipped;
 *     a splat that would take T below t_min ends the pixel and is not blended.
 *   - depth output is sum_i w_i z_i (camera z, not divided by alpha); the normal
 *     output is sum_i w_i n_i; colour adds T_final * background.
 *   - pixel (x, y) is sampled at (x + 0.5, y + 0.5).
 *   - the depth order and the near-plane test use a float32 camera depth
 *     z32 = ((r20*x + r21*y) + r22*z) + t2, every operation rounded to float32,
 *     ties broken by splat index: both sides take this integer decision in the
 *     kernel's precision, so the order is identical.
 *
 * Per-pixel borderline flags mark decisions that FP32 and FP64 may take
 * differently (support edge, alpha_min edge, t_min edge, normal facing edge),
 * and pixels whose sample point lies within 0.25 px of the centre of a blended
 * splat with beta < 2, where the falloff of Eq. 3 has a cusp (its mean-position
 * gradient keeps a finite size but takes its direction from a sub-pixel offset
 * that float32 screen coordinates do not resolve).
 *
 * For large images the per-pixel loop may walk a cell index instead of every
 * visible splat; that index only leaves out splats whose step of the loop does
 * nothing (see below), so both give the same result bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float viewmat[12]; /* row-major 3x4 [R | t], world -> camera */
    float znear;
} orc_camera;

typedef struct {
    int32_t sh_degree; /* -1: colour given as RGB; 0..3: SH coefficients */
    int32_t phi_mode;  /* 0 off, 1 centred, 2 literal Eq. 7 */
    float rho, lowpass, alpha_min, alpha_max, t_min, jac_clamp;
    float bg[3];
    float flag_eps; /* relative width of the borderline bands */
    int32_t cell;   /* 0: every pixel walks every visible splat; > 0: pixel cells of cell x cell (see
                       the cell index below) */
    float shift[2]; /* offset of the sample points from the pixel centres (0, 0 for the method; the
                       parity tests move them by the float32 rounding of the screen centres to see
                       how far the gradient moves with it) */
} orc_config;

/* Projected state of one splat in one view (FP64 except z32). */
typedef struct {
    int visible;
    float z32;
    double u, v, z;
    double tx, ty, tz;
    double S[3];     /* Sigma' (00, 01, 11) including the low-pass term */
    double conic[3]; /* (a, b, c): Q = a dx^2 + 2 b dx dy + c dy^2 */
    double qcut;
    double beta, opacity;
    double rgb[3];
    double normal[3];
    double facing; /* n . (campos - mu) / |campos - mu| before the sign flip */
    double du, dv; /* bound on the float32 rounding of (u, v) on the GPU side (pixels), for the flags */
    double qflag;  /* Q beyond which the splat neither passes the support test nor sets a flag */
} orc_splat;

/* ------------------------------------------------------------------ helpers */

static int n_sh_coeffs(int deg) { return deg < 0 ? 1 : (deg + 1) * (deg + 1); }

/* Rotation matrix of the unit quaternion qn = (w, x, y, z), row-major. */
static void quat_to_rot(const double qn[4], double R[9]) {
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* phi(beta) of Eq. 7 and its derivative, by mode. */
static double phi_of_beta(double beta, double rho, int mode, double *dphi) {
    double arg, s;
    if (mode == 0) { *dphi = 0.0; return 1.0; }
    arg = (mode == 1) ? rho * (beta - 2.0) : (rho * beta - 2.0 * beta);
    s = 1.0 / (1.0 + exp(-arg));
    *dphi = 2.0 * s * (1.0 - s) * ((mode == 1) ? rho : (rho - 2.0));
    return 2.0 * s;
}

/* ---------------------------------------------------- real spherical harmonics
 * Y_lm(d) for unit d = (x, y, z), l <= 3, ordered (l, m = -l..l), with the
 * Condon-Shortley phase:
 *   m > 0: sqrt2 K_l^m Pt_l^m(z) Re((x + i y)^m)
 *   m < 0: sqrt2 K_l^|m| Pt_l^|m|(z) Im((x + i y)^|m|)
 *   m = 0: K_l^0 Pt_l^0(z)
 * where K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) and Pt_l^m = P_l^m / sin^m(theta),
 * a polynomial in z obtained from the associated-Legendre recurrences. The
 * gradient is that of this polynomial extension in (x, y, z). */
static double factorial(int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; }

static void legendre_tilde(int l, int m, double z, double *p, double *dp) {
    /* Pt_m^m = (-1)^m (2m-1)!!, Pt_{m+1}^m = (2m+1) z Pt_m^m,
       (l-m) Pt_l^m = (2l-1) z Pt_{l-1}^m - (l+m-1) Pt_{l-2}^m */
    double dfact = 1.0;
    for (int i = 1; i <= 2 * m - 1; i += 2) dfact *= i;
    double pmm = ((m & 1) ? -1.0 : 1.0) * dfact, dpmm = 0.0;
    if (l == m) { *p = pmm; *dp = dpmm; return; }
    double p1 = (2 * m + 1) * z * pmm, dp1 = (2 * m + 1) * pmm;
    if (l == m + 1) { *p = p1; *dp = dp1; return; }
    double p0 = pmm, dp0 = dpmm;
    for (int ll = m + 2; ll <= l; ++ll) {
        double p2 = ((2 * ll - 1) * z * p1 - (ll + m - 1) * p0) / (ll - m);
        double dp2 = ((2 * ll - 1) * (p1 + z * dp1) - (ll + m - 1) * dp0) / (ll - m);
        p0 = p1; dp0 = dp1; p1 = p2; dp1 = dp2;
    }
    *p = p1; *dp = dp1;
}

static void sh_basis(int deg, const double d[3], double *Y, double (*dY)[3]) {
    double x = d[0], y = d[1], z = d[2];
    int k = 0;
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m, ++k) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            double P, dP;
            legendre_tilde(l, am, z, &P, &dP);
            /* (x + i y)^am and its derivative m (x + i y)^(am-1) */
            double re = 1.0, im = 0.0, re1 = 1.0, im1 = 0.0;
            for (int i = 0; i < am; ++i) {
                if (i == am - 1) { re1 = re; im1 = im; }
                double nr = re * x - im * y, ni = re * y + im * x;
                re = nr; im = ni;
            }
            if (m == 0) {
                Y[k] = K * P;
                if (dY) { dY[k][0] = 0.0; dY[k][1] = 0.0; dY[k][2] = K * dP; }
            } else {
                double c = sqrt(2.0) * K;
                /* d/dx (x+iy)^m = m (x+iy)^(m-1); d/dy = i m (x+iy)^(m-1) */
                double drx = am * re1, dix = am * im1;   /* d(re), d(im) / dx */
                double dry = -am * im1, diy = am * re1;  /* d(re), d(im) / dy */
                double A = (m > 0) ? re : im;
                double dAx = (m > 0) ? drx : dix, dAy = (m > 0) ? dry : diy;
                Y[k] = c * P * A;
                if (dY) { dY[k][0] = c * P * dAx; dY[k][1] = c * P * dAy; dY[k][2] = c * dP * A; }
            }
        }
    }
}

/* float32 camera depth with a fixed operation order, each step rounded. */
static float depth32(const float vm[12], const double mu[3]) {
    volatile float x = (float)mu[0], y = (float)mu[1], z = (float)mu[2];
    volatile float a = vm[8] * x;
    volatile float b = vm[9] * y;
    volatile float s = a + b;
    volatile float c = vm[10] * z;
    volatile float s2 = s + c;
    volatile float r = s2 + vm[11];
    return r;
}

/* Squared Mahalanobis radius beyond which a splat changes no pixel's loop: it passes the support
 * test only where Q <= qcut, and sets the support-edge flag only where Q <= q* + dQ with
 * q* = qcut (1 + flag_eps) and dQ as in render_pixel. With r = sqrt(Q), |C d| <= sqrt(lam) r (lam
 * the largest eigenvalue of the conic C) and dQ <= 2 sqrt2 delta |C d| + 2^-20 Q (delta =
 * max(du, dv)), both need (1 - 2^-20) r^2 - 2 sqrt2 delta sqrt(lam) r - q* <= 0, i.e. r <= r_max;
 * returns r_max^2 (1 + 1e-9). */
static double flag_radius2(const orc_splat *s, double eps) {
    const double c0 = s->conic[0], c1 = s->conic[1], c2 = s->conic[2];
    const double lam = 0.5 * (c0 + c2) + sqrt(0.25 * (c0 - c2) * (c0 - c2) + c1 * c1);
    const double dl = s->du > s->dv ? s->du : s->dv, k = 1.0 - ldexp(1.0, -20);
    const double rmax = (sqrt(2.0 * lam) * dl + sqrt(2.0 * lam * dl * dl + k * s->qcut * (1.0 + eps))) / k;
    return rmax * rmax * (1.0 + 1e-9);
}

/* ------------------------------------------------------------ S1 - S4 */
static void project_splat(const double *pos_op, const double *lsb, const double *quat, const double *color,
                          const orc_camera *cam, const orc_config *cfg, orc_splat *s) {
    memset(s, 0, sizeof(*s));
    const double mu[3] = {pos_op[0], pos_op[1], pos_op[2]};
    const double op = pos_op[3], beta = lsb[3];
    s->opacity = op;
    s->beta = beta;
    s->z32 = depth32(cam->viewmat, mu);
    if (!(s->z32 > cam->znear)) return;
    if (!(op >= (double)cfg->alpha_min)) return;

    /* S1: Sigma = R diag(s'^2) R^T with s' = phi(beta) exp(l) */
    double qn[4], qnorm = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    for (int i = 0; i < 4; ++i) qn[i] = quat[i] / qnorm;
    double R[9];
    quat_to_rot(qn, R);
    double dphi, phi = phi_of_beta(beta, cfg->rho, cfg->phi_mode, &dphi);
    double sp[3];
    for (int k = 0; k < 3; ++k) sp[k] = phi * exp(lsb[k]);
    double Sig[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[i * 3 + k] * sp[k] * sp[k] * R[j * 3 + k];
            Sig[i * 3 + j] = acc;
        }

    /* S2: camera transform, Jacobian of the perspective map, EWA covariance */
    double W[9], tw[3], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) W[i * 3 + j] = cam->viewmat[i * 4 + j];
        tw[i] = cam->viewmat[i * 4 + 3];
    }
    for (int i = 0; i < 3; ++i) t[i] = W[i * 3 + 0] * mu[0] + W[i * 3 + 1] * mu[1] + W[i * 3 + 2] * mu[2] + tw[i];
    s->tx = t[0]; s->ty = t[1]; s->tz = t[2];
    const double fx = cam->fx, fy = cam->fy;
    const double limx = cfg->jac_clamp * 0.5 * cam->width / fx, limy = cfg->jac_clamp * 0.5 * cam->height / fy;
    double rx = t[0] / t[2], ry = t[1] / t[2];
    rx = rx < -limx ? -limx : (rx > limx ? limx : rx);
    ry = ry < -limy ? -limy : (ry > limy ? limy : ry);
    double txc = rx * t[2], tyc = ry * t[2];
    double J[6] = {fx / t[2], 0.0, -fx * txc / (t[2] * t[2]), 0.0, fy / t[2], -fy * tyc / (t[2] * t[2])};
    double T[6]; /* T = J W */
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) T[i * 3 + j] = J[i * 3 + 0] * W[0 * 3 + j] + J[i * 3 + 1] * W[1 * 3 + j] + J[i * 3 + 2] * W[2 * 3 + j];
    double M[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += T[i * 3 + k] * Sig[k * 3 + l] * T[j * 3 + l];
            M[i * 2 + j] = acc;
        }
    M[0] += cfg->lowpass; M[3] += cfg->lowpass;
    s->S[0] = M[0]; s->S[1] = 0.5 * (M[1] + M[2]); s->S[2] = M[3];
    double det = s->S[0] * s->S[2] - s->S[1] * s->S[1];
    if (!(det > 0)) return;
    s->conic[0] = s->S[2] / det; s->conic[1] = -s->S[1] / det; s->conic[2] = s->S[0] / det;
    s->u = fx * t[0] / t[2] + cam->cx;
    s->v = fy * t[1] / t[2] + cam->cy;
    s->z = t[2];
    /* First-order bound on the float32 rounding of u, v as the GPU computes them (t_i as a
       float32 dot product plus translation, then fx t_x / t_z + c_x): each t_i carries at most
       2^-22 (sum_j |W_ij mu_j| + |t_i|), and u carries fx (e_x + |t_x / t_z| e_z) / t_z plus
       2^-22 (|u| + |u - c_x|) from its own operations. Only the borderline flags use it. */
    {
        double et[3];
        for (int i = 0; i < 3; ++i)
            et[i] = ldexp(fabs(W[i * 3 + 0] * mu[0]) + fabs(W[i * 3 + 1] * mu[1]) + fabs(W[i * 3 + 2] * mu[2]) +
                          fabs(tw[i]), -22);
        s->du = fx * (et[0] + fabs(t[0] / t[2]) * et[2]) / t[2] + ldexp(fabs(s->u) + fabs(s->u - cam->cx), -22);
        s->dv = fy * (et[1] + fabs(t[1] / t[2]) * et[2]) / t[2] + ldexp(fabs(s->v) + fabs(s->v - cam->cy), -22);
    }

    /* S3: exact support of exp(-1/2 Q^(beta/2)) >= alpha_min / o */
    s->qcut = pow(2.0 * log(op / (double)cfg->alpha_min), 2.0 / beta);

    /* S4: colour */
    double campos[3];
    for (int j = 0; j < 3; ++j) campos[j] = -(W[0 * 3 + j] * tw[0] + W[1 * 3 + j] * tw[1] + W[2 * 3 + j] * tw[2]);
    if (cfg->sh_degree < 0) {
        for (int c = 0; c < 3; ++c) s->rgb[c] = color[c];
    } else {
        double dv[3] = {mu[0] - campos[0], mu[1] - campos[1], mu[2] - campos[2]};
        double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        for (int j = 0; j < 3; ++j) dv[j] /= dn;
        double Y[16];
        int K = n_sh_coeffs(cfg->sh_degree);
        sh_basis(cfg->sh_degree, dv, Y, NULL);
        for (int c = 0; c < 3; ++c) {
            double acc = 0.5;
            for (int k = 0; k < K; ++k) acc += color[k * 3 + c] * Y[k];
            s->rgb[c] = acc > 0 ? acc : 0.0;
        }
    }
    /* normal: column of R for the smallest scale (ties -> lowest index), facing the camera */
    int ks = 0;
    if (lsb[1] < lsb[ks]) ks = 1;
    if (lsb[2] < lsb[ks]) ks = 2;
    double n[3] = {R[0 * 3 + ks], R[1 * 3 + ks], R[2 * 3 + ks]};
    double vc[3] = {campos[0] - mu[0], campos[1] - mu[1], campos[2] - mu[2]};
    double vcn = sqrt(vc[0] * vc[0] + vc[1] * vc[1] + vc[2] * vc[2]);
    double f = (n[0] * vc[0] + n[1] * vc[1] + n[2] * vc[2]) / vcn;
    s->facing = f;
    double sg = (f < 0) ? -1.0 : 1.0;
    for (int j = 0; j < 3; ++j) s->normal[j] = sg * n[j];
    s->qflag = flag_radius2(s, cfg->flag_eps);
    s->visible = 1;
}

/* ------------------------------------------------------------ ordering (S5) */
typedef struct { uint32_t key; int32_t id; } orc_order;

static int cmp_order(const void *a, const void *b) {
    const orc_order *x = (const orc_order *)a, *y = (const orc_order *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

static int32_t *visible_order(int n, const orc_splat *sp, int *n_vis) {
    orc_order *tmp = (orc_order *)malloc(sizeof(orc_order) * (size_t)(n > 0 ? n : 1));
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (sp[i].visible) {
            uint32_t bits;
            memcpy(&bits, &sp[i].z32, 4);
            tmp[m].key = bits; tmp[m].id = i; ++m;
        }
    qsort(tmp, (size_t)m, sizeof(orc_order), cmp_order);
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    for (int i = 0; i < m; ++i) ord[i] = tmp[i].id;
    free(tmp);
    *n_vis = m;
    return ord;
}

/* ------------------------------------------------------------ cell index
 * The image is cut into cells of c x c pixels. Each cell lists, in the depth
 * order of S5, every visible splat whose widened support box reaches a pixel
 * centre of the cell. A splat changes a pixel's loop only where Q <= qflag
 * (flag_radius2). The box of the ellipse Q <= q (Q = d^T Sigma'^-1 d) is
 * |dx| <= sqrt(q Sigma'_00), |dy| <= sqrt(q Sigma'_11), taken at q = qflag and
 * widened by 1e-6 px. A splat that a pixel's cell does not list is therefore a no-op step
 * of that pixel's loop, and the loop over the cell's list gives the result of
 * the loop over all splats bit for bit. */
typedef struct {
    int c, ncx, ncy;
    size_t *start; /* ncx * ncy + 1 */
    int32_t *ids;
} orc_cells;

static int cell_box(const orc_splat *s, const orc_camera *cam, double eps, const float shift[2], int c, int *cx0,
                    int *cx1, int *cy0, int *cy1) {
    (void)eps;
    const double q = s->qflag;
    const double ex = sqrt(s->S[0] * q) + 1e-6 + fabs(shift[0]), ey = sqrt(s->S[2] * q) + 1e-6 + fabs(shift[1]);
    /* pixel x (sampled at x + 0.5 + shift, |shift| added to ex above) can be in the support iff
       |x + 0.5 - u| <= ex */
    double x0 = ceil(s->u - ex - 0.5), x1 = floor(s->u + ex - 0.5);
    double y0 = ceil(s->v - ey - 0.5), y1 = floor(s->v + ey - 0.5);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > cam->width - 1) x1 = cam->width - 1;
    if (y1 > cam->height - 1) y1 = cam->height - 1;
    if (!(x0 <= x1 && y0 <= y1)) return 0;
    *cx0 = (int)x0 / c; *cx1 = (int)x1 / c; *cy0 = (int)y0 / c; *cy1 = (int)y1 / c;
    return 1;
}

static void build_cells(const int32_t *ord, int nv, const orc_splat *sp, const orc_camera *cam, double eps,
                        const float shift[2], int c, orc_cells *out) {
    out->c = c;
    out->ncx = (cam->width + c - 1) / c;
    out->ncy = (cam->height + c - 1) / c;
    const size_t nc = (size_t)out->ncx * out->ncy;
    out->start = (size_t *)calloc(nc + 1, sizeof(size_t));
    for (int k = 0; k < nv; ++k) {
        int cx0, cx1, cy0, cy1;
        if (!cell_box(&sp[ord[k]], cam, eps, shift, c, &cx0, &cx1, &cy0, &cy1)) continue;
        for (int cy = cy0; cy <= cy1; ++cy)
            for (int cx = cx0; cx <= cx1; ++cx) out->start[(size_t)cy * out->ncx + cx + 1]++;
    }
    for (size_t i = 0; i < nc; ++i) out->start[i + 1] += out->start[i];
    out->ids = (int32_t *)malloc(sizeof(int32_t) * (out->start[nc] > 0 ? out->start[nc] : 1));
    size_t *fill = (size_t *)malloc(sizeof(size_t) * (nc > 0 ? nc : 1));
    memcpy(fill, out->start, sizeof(size_t) * nc);
    for (int k = 0; k < nv; ++k) { /* in depth order, so every list keeps it */
        int cx0, cx1, cy0, cy1;
        if (!cell_box(&sp[ord[k]], cam, eps, shift, c, &cx0, &cx1, &cy0, &cy1)) continue;
        for (int cy = cy0; cy <= cy1; ++cy)
            for (int cx = cx0; cx <= cx1; ++cx) out->ids[fill[(size_t)cy * out->ncx + cx]++] = ord[k];
    }
    free(fill);
}

/* The splats pixel (x, y) walks: its cell's list, or all visible splats. */
static const int32_t *pixel_list(const orc_cells *cells, const int32_t *ord, int nv, int x, int y, int *len) {
    if (!cells) { *len = nv; return ord; }
    const size_t ci = (size_t)(y / cells->c) * cells->ncx + (size_t)(x / cells->c);
    *len = (int)(cells->start[ci + 1] - cells->start[ci]);
    return cells->ids + cells->start[ci];
}

static void free_cells(orc_cells *cells) {
    if (!cells) return;
    free(cells->start);
    free(cells->ids);
}

/* ------------------------------------------------------------ S6, one pixel */
typedef struct {
    double color[3], depth, alpha, normal[3], T;
    int ncontrib, last_id, flags;
} orc_pixel;

enum { FLAG_SUPPORT = 1, FLAG_ALPHA_MIN = 2, FLAG_T_MIN = 4, FLAG_FACING = 8, FLAG_CUSP = 16 };

static double falloff(double Q, double beta) { return exp(-0.5 * pow(Q, 0.5 * beta)); }

/* Borderline bands. A decision is flagged when float32 may take it the other way: Q against
 * qcut within eps qcut plus dQ, the change of Q under the float32 rounding (du, dv) of the
 * splat's screen centre, dQ = 2 (|m_x| du + |m_y| dv) with m = C d, plus 2^-20 Q for the conic's
 * own rounding; alpha against alpha_min within eps alpha_min plus the matching d alpha =
 * alpha (beta / 4) p dQ / Q; the transmittance against t_min within (eps + rT) t_min, rT the
 * relative error it has gathered: sum of d alpha / (1 - alpha) over the blended splats and
 * 2^-21 (1 + p) for each one's float32 falloff and product. */
static void render_pixel(const int32_t *ord, int nv, const orc_splat *sp, double px, double py,
                         const orc_config *cfg, orc_pixel *out) {
    double T = 1.0, C[3] = {0, 0, 0}, D = 0, N[3] = {0, 0, 0}, rT = 0.0;
    int cnt = 0, last = -1, flags = 0;
    const double eps = cfg->flag_eps;
    const double amin = cfg->alpha_min, amax = cfg->alpha_max, tmin = cfg->t_min;
    for (int k = 0; k < nv; ++k) {
        const orc_splat *s = &sp[ord[k]];
        double dx = px - s->u, dy = py - s->v;
        double Q = s->conic[0] * dx * dx + 2.0 * s->conic[1] * dx * dy + s->conic[2] * dy * dy;
        if (Q > s->qflag) continue; /* outside the support and every band: a no-op step */
        const double mx = s->conic[0] * dx + s->conic[1] * dy, my = s->conic[1] * dx + s->conic[2] * dy;
        const double dQ = 2.0 * (fabs(mx) * s->du + fabs(my) * s->dv) + ldexp(fabs(Q), -20);
        if (fabs(Q - s->qcut) <= eps * s->qcut + dQ) flags |= FLAG_SUPPORT;
        if (Q > s->qcut) continue;
        double G = falloff(Q, s->beta);
        double a = s->opacity * G;
        if (a > amax) a = amax;
        const double p = pow(Q, 0.5 * s->beta);
        const double da = Q > 0 ? a * 0.25 * s->beta * p * dQ / Q : 0.0;
        if (fabs(a - amin) <= eps * amin + da) flags |= FLAG_ALPHA_MIN;
        if (a < amin) continue;
        double Tn = T * (1.0 - a);
        const double rTn = rT + da / (1.0 - a) + ldexp(1.0 + p, -21);
        if (fabs(Tn - tmin) <= (eps + rTn) * tmin) flags |= FLAG_T_MIN;
        if (Tn < tmin) break;
        rT = rTn;
        double w = a * T;
        for (int c = 0; c < 3; ++c) C[c] += w * s->rgb[c];
        D += w * s->z;
        for (int c = 0; c < 3; ++c) N[c] += w * s->normal[c];
        if (fabs(s->facing) <= eps) flags |= FLAG_FACING;
        if (s->beta < 2.0 && dx * dx + dy * dy < 0.0625) flags |= FLAG_CUSP;
        T = Tn;
        ++cnt;
        last = ord[k];
    }
    for (int c = 0; c < 3; ++c) out->color[c] = C[c] + T * cfg->bg[c];
    out->depth = D;
    out->alpha = 1.0 - T;
    for (int c = 0; c < 3; ++c) out->normal[c] = N[c];
    out->T = T;
    out->ncontrib = cnt;
    out->last_id = last;
    out->flags = flags;
}

/* -------------------------------------------------- exported: preprocess */
int orc_preprocess(int n, const double *pos_op, const double *lsb, const double *quat, const double *color,
                   const orc_camera *cam, const orc_config *cfg,
                   int32_t *visible, float *z32, double *uvz, double *cov2d, double *conic, double *qcut,
                   double *rgb, double *normal, double *duv) {
    int K3 = 3 * n_sh_coeffs(cfg->sh_degree);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        orc_splat s;
        project_splat(pos_op + 4 * i, lsb + 4 * i, quat + 4 * i, color + (size_t)K3 * i, cam, cfg, &s);
        visible[i] = s.visible;
        z32[i] = s.z32;
        uvz[3 * i + 0] = s.u; uvz[3 * i + 1] = s.v; uvz[3 * i + 2] = s.z;
        for (int j = 0; j < 3; ++j) {
            cov2d[3 * i + j] = s.S[j]; conic[3 * i + j] = s.conic[j];
            rgb[3 * i + j] = s.rgb[j]; normal[3 * i + j] = s.normal[j];
        }
        qcut[i] = s.qcut;
        if (duv) { duv[2 * i] = s.du; duv[2 * i + 1] = s.dv; }
    }
    return 0;
}

static orc_splat *project_all(int n, const double *pos_op, const double *lsb, const double *quat,
                              const double *color, const orc_camera *cam, const orc_config *cfg) {
    int K3 = 3 * n_sh_coeffs(cfg->sh_degree);
    orc_splat *sp = (orc_splat *)malloc(sizeof(orc_splat) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        project_splat(pos_op + 4 * i, lsb + 4 * i, quat + 4 * i, color + (size_t)K3 * i, cam, cfg, &sp[i]);
    return sp;
}

/* -------------------------------------------------- exported: forward
 * pix: npix (x, y) pairs, or NULL for the whole image in row-major order. */
int orc_render(int n, const double *pos_op, const double *lsb, const double *quat, const double *color,
               const orc_camera *cam, const orc_config *cfg, int npix, const int32_t *pix,
               double *color_out, double *depth_out, double *alpha_out, double *normal_out, double *T_out,
               int32_t *ncontrib, int32_t *last_id, int32_t *flags) {
    orc_splat *sp = project_all(n, pos_op, lsb, quat, color, cam, cfg);
    int nv;
    int32_t *ord = visible_order(n, sp, &nv);
    orc_cells cells_, *cells = NULL;
    if (cfg->cell > 0) { build_cells(ord, nv, sp, cam, cfg->flag_eps, cfg->shift, cfg->cell, &cells_); cells = &cells_; }
#pragma omp parallel for schedule(dynamic, 8)
    for (int p = 0; p < npix; ++p) {
        int x = pix ? pix[2 * p] : p % cam->width;
        int y = pix ? pix[2 * p + 1] : p / cam->width;
        orc_pixel o;
        int len;
        const int32_t *lst = pixel_list(cells, ord, nv, x, y, &len);
        render_pixel(lst, len, sp, x + 0.5 + cfg->shift[0], y + 0.5 + cfg->shift[1], cfg, &o);
        for (int c = 0; c < 3; ++c) { color_out[3 * p + c] = o.color[c]; normal_out[3 * p + c] = o.normal[c]; }
        depth_out[p] = o.depth; alpha_out[p] = o.alpha; T_out[p] = o.T;
        ncontrib[p] = o.ncontrib; last_id[p] = o.last_id; flags[p] = o.flags;
    }
    free_cells(cells);
    free(ord);
    free(sp);
    return 0;
}

/* -------------------------------------------------- S7: gradient of one pixel
 * Accumulates the screen-space gradient of every blended splat into g2d
 * (16 doubles per splat: u, v, a, b, c, opacity, beta, z, r, g, b, -, nx, ny, nz, -).
 * Front-to-back replay: with w_i = alpha_i T_i and the final value X (colour incl.
 * T_final * bg, depth, normal) the part behind splat i is X - sum_{j<=i} w_j x_j, so
 *   dX/dalpha_i = T_i x_i - (X - sum_{j<=i} w_j x_j) / (1 - alpha_i),
 *   dA/dalpha_i = T_final / (1 - alpha_i)  (A = 1 - T_final).               */
static void backward_pixel(const int32_t *ord, int nv, const orc_splat *sp, double px, double py,
                           const orc_config *cfg, const double gC[3], double gD, double gA, const double gN[3],
                           double *g2d) {
    orc_pixel fwd;
    render_pixel(ord, nv, sp, px, py, cfg, &fwd);
    const double amin = cfg->alpha_min, amax = cfg->alpha_max;
    double T = 1.0, Cacc[3] = {0, 0, 0}, Dacc = 0, Nacc[3] = {0, 0, 0};
    int blended = 0;
    for (int k = 0; k < nv && blended < fwd.ncontrib; ++k) {
        int id = ord[k];
        const orc_splat *s = &sp[id];
        double dx = px - s->u, dy = py - s->v;
        double a_ = s->conic[0], b_ = s->conic[1], c_ = s->conic[2];
        double Q = a_ * dx * dx + 2.0 * b_ * dx * dy + c_ * dy * dy;
        if (Q > s->qcut) continue;
        double hb = 0.5 * s->beta;
        double p = pow(Q, hb);
        double G = exp(-0.5 * p);
        double araw = s->opacity * G;
        double a = araw > amax ? amax : araw;
        if (a < amin) continue;
        ++blended;
        double w = a * T;
        for (int c = 0; c < 3; ++c) Cacc[c] += w * s->rgb[c];
        Dacc += w * s->z;
        for (int c = 0; c < 3; ++c) Nacc[c] += w * s->normal[c];
        double inv1ma = 1.0 / (1.0 - a);
        double dalpha = 0.0;
        for (int c = 0; c < 3; ++c) dalpha += gC[c] * (T * s->rgb[c] - (fwd.color[c] - Cacc[c]) * inv1ma);
        dalpha += gD * (T * s->z - (fwd.depth - Dacc) * inv1ma);
        for (int c = 0; c < 3; ++c) dalpha += gN[c] * (T * s->normal[c] - (fwd.normal[c] - Nacc[c]) * inv1ma);
        dalpha += gA * fwd.T * inv1ma;
        double *g = g2d + 16 * (size_t)id;
        double go = 0, gG = 0;
        if (araw < amax) { go = dalpha * G; gG = dalpha * s->opacity; }
        double dGdQ = 0, dGdb = 0;
        if (Q > 0) { dGdQ = -0.5 * hb * p / Q * G; dGdb = -0.25 * p * log(Q) * G; }
        double gQ = gG * dGdQ;
        double contrib[16] = {
            gQ * -(2 * a_ * dx + 2 * b_ * dy), gQ * -(2 * b_ * dx + 2 * c_ * dy),
            gQ * dx * dx, gQ * 2 * dx * dy, gQ * dy * dy,
            go, gG * dGdb, gD * w,
            gC[0] * w, gC[1] * w, gC[2] * w, 0.0,
            gN[0] * w, gN[1] * w, gN[2] * w, 0.0};
        for (int j = 0; j < 16; ++j) {
#pragma omp atomic
            g[j] += contrib[j];
        }
        T *= (1.0 - a);
    }
}

/* -------------------------------------------------- S8: chain rule of one splat */
static void backprop_splat(const double *pos_op, const double *lsb, const double *quat, const double *color,
                           const orc_camera *cam, const orc_config *cfg, const orc_splat *s, const double *g2,
                           double *g_pos_op, double *g_lsb, double *g_quat, double *g_color) {
    const double mu[3] = {pos_op[0], pos_op[1], pos_op[2]};
    const double beta = lsb[3];
    double qnorm = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    double qn[4];
    for (int i = 0; i < 4; ++i) qn[i] = quat[i] / qnorm;
    double R[9];
    quat_to_rot(qn, R);
    double dphi, phi = phi_of_beta(beta, cfg->rho, cfg->phi_mode, &dphi);
    double es[3], sp[3];
    for (int k = 0; k < 3; ++k) { es[k] = exp(lsb[k]); sp[k] = phi * es[k]; }
    double Sig[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[i * 3 + k] * sp[k] * sp[k] * R[j * 3 + k];
            Sig[i * 3 + j] = acc;
        }
    double W[9], tw[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) W[i * 3 + j] = cam->viewmat[i * 4 + j];
        tw[i] = cam->viewmat[i * 4 + 3];
    }
    const double tx = s->tx, ty = s->ty, tz = s->tz;
    const double fx = cam->fx, fy = cam->fy;
    const double limx = cfg->jac_clamp * 0.5 * cam->width / fx, limy = cfg->jac_clamp * 0.5 * cam->height / fy;
    double rx = tx / tz, ry = ty / tz;
    int clx = (rx < -limx) || (rx > limx), cly = (ry < -limy) || (ry > limy);
    rx = rx < -limx ? -limx : (rx > limx ? limx : rx);
    ry = ry < -limy ? -limy : (ry > limy ? limy : ry);
    double txc = rx * tz, tyc = ry * tz;
    double J[6] = {fx / tz, 0.0, -fx * txc / (tz * tz), 0.0, fy / tz, -fy * tyc / (tz * tz)};
    double T[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) T[i * 3 + j] = J[i * 3 + 0] * W[0 * 3 + j] + J[i * 3 + 1] * W[1 * 3 + j] + J[i * 3 + 2] * W[2 * 3 + j];

    /* conic -> Sigma' : G_M = -C G_C C, with G_C symmetric (b is shared) */
    const double *C = s->conic;
    double Cm[4] = {C[0], C[1], C[1], C[2]};
    double GC[4] = {g2[2], 0.5 * g2[3], 0.5 * g2[3], g2[4]};
    double tmp[4], GM[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) tmp[i * 2 + j] = GC[i * 2 + 0] * Cm[0 * 2 + j] + GC[i * 2 + 1] * Cm[1 * 2 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) GM[i * 2 + j] = -(Cm[i * 2 + 0] * tmp[0 * 2 + j] + Cm[i * 2 + 1] * tmp[1 * 2 + j]);
    /* Sigma' = T Sigma T^T: G_Sigma = T^T G_M T, G_T = 2 G_M T Sigma */
    double GS[9], GT[6], TS[6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) acc += T[a * 3 + i] * GM[a * 2 + b] * T[b * 3 + j];
            GS[i * 3 + j] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += T[i * 3 + k] * Sig[k * 3 + j];
            TS[i * 3 + j] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) GT[i * 3 + j] = 2.0 * (GM[i * 2 + 0] * TS[0 * 3 + j] + GM[i * 2 + 1] * TS[1 * 3 + j]);
    /* T = J W: G_J = G_T W^T */
    double GJ[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) GJ[i * 3 + j] = GT[i * 3 + 0] * W[j * 3 + 0] + GT[i * 3 + 1] * W[j * 3 + 1] + GT[i * 3 + 2] * W[j * 3 + 2];
    double gt[3] = {0, 0, 0};
    gt[2] += -fx / (tz * tz) * GJ[0] - fy / (tz * tz) * GJ[4];
    if (!clx) { gt[0] += -fx / (tz * tz) * GJ[2]; gt[2] += 2.0 * fx * tx / (tz * tz * tz) * GJ[2]; }
    else gt[2] += fx * txc / (tz * tz * tz) * GJ[2];
    if (!cly) { gt[1] += -fy / (tz * tz) * GJ[5]; gt[2] += 2.0 * fy * ty / (tz * tz * tz) * GJ[5]; }
    else gt[2] += fy * tyc / (tz * tz * tz) * GJ[5];
    /* mean: u = fx tx/tz + cx, v = fy ty/tz + cy; depth value z = tz */
    gt[0] += fx / tz * g2[0]; gt[2] += -fx * tx / (tz * tz) * g2[0];
    gt[1] += fy / tz * g2[1]; gt[2] += -fy * ty / (tz * tz) * g2[1];
    gt[2] += g2[7];
    double gmu[3];
    for (int j = 0; j < 3; ++j) gmu[j] = W[0 * 3 + j] * gt[0] + W[1 * 3 + j] * gt[1] + W[2 * 3 + j] * gt[2];

    /* Sigma = R D R^T, D = diag(s'^2): G_R = 2 G_Sigma R D, g_D = diag(R^T G_Sigma R) */
    double GR[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += GS[i * 3 + j] * R[j * 3 + k];
            GR[i * 3 + k] = 2.0 * acc * sp[k] * sp[k];
        }
    double gbeta = g2[6];
    for (int k = 0; k < 3; ++k) {
        double gD = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) gD += R[i * 3 + k] * GS[i * 3 + j] * R[j * 3 + k];
        double gsp = 2.0 * sp[k] * gD;
        g_lsb[k] += gsp * sp[k];
        gbeta += gsp * dphi * es[k];
    }
    g_lsb[3] += gbeta;
    /* normal: n = sign * R[:, k*] */
    int ks = 0;
    if (lsb[1] < lsb[ks]) ks = 1;
    if (lsb[2] < lsb[ks]) ks = 2;
    double sg = (s->facing < 0) ? -1.0 : 1.0;
    for (int i = 0; i < 3; ++i) GR[i * 3 + ks] += sg * g2[12 + i];
    /* R(qn) -> qn -> q */
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    double gq[4];
    gq[0] = 2 * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    gq[1] = 2 * (y * GR[1] + z * GR[2] + y * GR[3] - 2 * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2 * x * GR[8]);
    gq[2] = 2 * (-2 * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2 * y * GR[8]);
    gq[3] = 2 * (-2 * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2 * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
    double dq = gq[0] * qn[0] + gq[1] * qn[1] + gq[2] * qn[2] + gq[3] * qn[3];
    for (int i = 0; i < 4; ++i) g_quat[i] += (gq[i] - qn[i] * dq) / qnorm;

    /* colour */
    if (cfg->sh_degree < 0) {
        for (int c = 0; c < 3; ++c) g_color[c] += g2[8 + c];
    } else {
        double campos[3];
        for (int j = 0; j < 3; ++j) campos[j] = -(W[0 * 3 + j] * tw[0] + W[1 * 3 + j] * tw[1] + W[2 * 3 + j] * tw[2]);
        double dv[3] = {mu[0] - campos[0], mu[1] - campos[1], mu[2] - campos[2]};
        double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        double d[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn};
        int K = n_sh_coeffs(cfg->sh_degree);
        double Y[16], dY[16][3];
        sh_basis(cfg->sh_degree, d, Y, dY);
        double gd[3] = {0, 0, 0};
        for (int c = 0; c < 3; ++c) {
            double pre = 0.5;
            for (int k = 0; k < K; ++k) pre += color[k * 3 + c] * Y[k];
            if (!(pre > 0)) continue;
            double gc = g2[8 + c];
            for (int k = 0; k < K; ++k) {
                g_color[k * 3 + c] += gc * Y[k];
                for (int j = 0; j < 3; ++j) gd[j] += gc * color[k * 3 + c] * dY[k][j];
            }
        }
        double dd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
        for (int j = 0; j < 3; ++j) gmu[j] += (gd[j] - d[j] * dd) / dn;
    }
    for (int j = 0; j < 3; ++j) g_pos_op[j] += gmu[j];
    g_pos_op[3] += g2[5];
}

/* -------------------------------------------------- exported: backward
 * Upstream gradients g_* are given per listed pixel (npix entries, colour and
 * normal interleaved as 3 per pixel). Outputs are ACCUMULATED into the caller's
 * arrays (zero them first); g2d (16 per splat) may be NULL. */
int orc_backward(int n, const double *pos_op, const double *lsb, const double *quat, const double *color,
                 const orc_camera *cam, const orc_config *cfg, int npix, const int32_t *pix,
                 const double *g_color, const double *g_depth, const double *g_alpha, const double *g_normal,
                 double *g2d_out, double *g_pos_op, double *g_lsb, double *g_quat, double *g_col) {
    orc_splat *sp = project_all(n, pos_op, lsb, quat, color, cam, cfg);
    int nv;
    int32_t *ord = visible_order(n, sp, &nv);
    double *g2d = (double *)calloc((size_t)16 * (size_t)(n > 0 ? n : 1), sizeof(double));
    orc_cells cells_, *cells = NULL;
    if (cfg->cell > 0) { build_cells(ord, nv, sp, cam, cfg->flag_eps, cfg->shift, cfg->cell, &cells_); cells = &cells_; }
#pragma omp parallel for schedule(dynamic, 8)
    for (int p = 0; p < npix; ++p) {
        int x = pix ? pix[2 * p] : p % cam->width;
        int y = pix ? pix[2 * p + 1] : p / cam->width;
        int len;
        const int32_t *lst = pixel_list(cells, ord, nv, x, y, &len);
        backward_pixel(lst, len, sp, x + 0.5 + cfg->shift[0], y + 0.5 + cfg->shift[1], cfg, g_color + 3 * p, g_depth[p], g_alpha[p],
                       g_normal + 3 * p, g2d);
    }
    free_cells(cells);
    int K3 = 3 * n_sh_coeffs(cfg->sh_degree);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        if (!sp[i].visible) continue;
        const double *g2 = g2d + 16 * (size_t)i;
        int any = 0;
        for (int j = 0; j < 16; ++j) any |= (g2[j] != 0.0);
        if (!any) continue;
        backprop_splat(pos_op + 4 * i, lsb + 4 * i, quat + 4 * i, color + (size_t)K3 * i, cam, cfg, &sp[i], g2,
                       g_pos_op + 4 * i, g_lsb + 4 * i, g_quat + 4 * i, g_col + (size_t)K3 * i);
    }
    if (g2d_out)
        for (size_t j = 0; j < (size_t)16 * n; ++j) g2d_out[j] += g2d[j];
    free(g2d);
    free(ord);
    free(sp);
    return 0;
}

/* -------------------------------------------------- exported: S8 alone
 * The chain rule of S1-S4 applied to a given per-splat screen-space gradient
 * g2d (16 per splat, the layout of orc_backward: u, v, conic a, b, c, opacity,
 * beta, z, r, g, b, -, nx, ny, nz, -). Outputs are ACCUMULATED. */
int orc_chain(int n, const double *pos_op, const double *lsb, const double *quat, const double *color,
              const orc_camera *cam, const orc_config *cfg, const double *g2d,
              double *g_pos_op, double *g_lsb, double *g_quat, double *g_col) {
    orc_splat *sp = project_all(n, pos_op, lsb, quat, color, cam, cfg);
    int K3 = 3 * n_sh_coeffs(cfg->sh_degree);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        if (!sp[i].visible) continue;
        backprop_splat(pos_op + 4 * i, lsb + 4 * i, quat + 4 * i, color + (size_t)K3 * i, cam, cfg, &sp[i],
                       g2d + 16 * (size_t)i, g_pos_op + 4 * i, g_lsb + 4 * i, g_quat + 4 * i, g_col + (size_t)K3 * i);
    }
    free(sp);
    return 0;
}

/* -------------------------------------------------- exported: SH basis (for pins) */
int orc_sh_basis(int deg, const double *d, double *Y, double *dY) {
    sh_basis(deg, d, Y, (double (*)[3])dY);
    return n_sh_coeffs(deg);
}

int orc_phi(double beta, double rho, int mode, double *phi, double *dphi) {
    *phi = phi_of_beta(beta, rho, mode, dphi);
    return 0;
}
