/*
 * FP64 CPU oracle for the forward 3D Gaussian Splatting rasterization of the
 * TIGAS backend.  TEST INFRASTRUCTURE ONLY: the product path never links,
 * loads or calls this file; only the tests, the smoke check and the timed
 * CPU baseline do.  It shares no code with the CUDA path.
 *
 * What it computes is the plain definition of the rendered frame, with no
 * tiling, sorting network or shared-memory staging:
 *   1. attribute activations of Sec. 5.1 (PLY Model and Primitives):
 *      scale = exp(s), opacity = sigmoid(logit), unit quaternion q/|q|;
 *   2. camera of Sec. 5.1 (Rendering Engine): R from azimuth/elevation,
 *      world->camera T = [R^T, -R^T t; 0, 1] and the pinhole projection
 *      lambda [u v 1]^T = K p_c with lambda = z_c;
 *   3. the tile-based 3DGS rasterizer the paper relies on (Sec. 4.1,
 *      Rendering Engine, citing Kerbl et al. 2023): EWA projection of
 *      Sigma = R_q S S^T R_q^T (Zwicker et al. 2001) with a 0.3 px^2 low-pass
 *      dilation, conic = inverse 2D covariance, 3-sigma radius and the 16x16
 *      tile rectangle that bounds a Gaussian's support, SH degree <= 3
 *      colour, and per-pixel front-to-back alpha compositing of every
 *      supported Gaussian in (depth, index) order, skipping alpha < 1/255
 *      and stopping before the Gaussian that would bring T below 1e-4.
 *
 * Readings where the paper is silent (the CUDA path takes the same ones;
 * the projection and compositing constants are those of the cited 3DGS
 * method, the pose and pixel conventions are this implementation's own):
 *   pose R = R_y(azimuth) R_x(elevation), camera axes x right, y down,
 *   z forward; pixel (i,j) sampled at (i+0.5, j+0.5); near plane z > 0.2;
 *   EWA guard band 1.3 x half-FOV; alpha cap 0.99; depth key = view z;
 *   real SH with the Condon-Shortley phase ordered m = -l..l; quaternion
 *   order (w,x,y,z); RGBA8 = floor(clamp(x,0,1)*255 + 0.5), A = 1 - T.
 *
 * Integer decisions (near cull, opacity cull, ceil of 3 sqrt(lambda), the
 * four tile-rect floors) are taken in FP64.  Each one also reports the range
 * of outcomes reachable within a small guard band around its threshold, so a
 * test can accept either outcome where FP32 rounding may legitimately flip
 * the decision (guard widths are arguments, not constants).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_TILE 16
#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------ camera */

/* R = R_y(az) R_x(el): columns are the camera's right, down, forward axes in
 * world coordinates.  World->camera rotation is R^T, translation -R^T t. */
void oracle_camera_rotation(double az, double el, double R[9]) {
    double ca = cos(az), sa = sin(az), ce = cos(el), se = sin(el);
    double Ry[9] = {ca, 0, sa, 0, 1, 0, -sa, 0, ca};
    double Rx[9] = {1, 0, 0, 0, ce, -se, 0, se, ce};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += Ry[r * 3 + k] * Rx[k * 3 + c];
            R[r * 3 + c] = s;
        }
}

/* 4x4 world->camera matrix T_{w->c} = [R^T, -R^T t; 0 1], row-major. */
void oracle_world_to_camera(double az, double el, const double t[3], double T[16]) {
    double R[9];
    oracle_camera_rotation(az, el, R);
    memset(T, 0, 16 * sizeof(double));
    for (int r = 0; r < 3; ++r) {
        double tr = 0;
        for (int c = 0; c < 3; ++c) {
            T[r * 4 + c] = R[c * 3 + r];       /* (R^T)_{rc} = R_{cr} */
            tr += R[c * 3 + r] * t[c];
        }
        T[r * 4 + 3] = -tr;
    }
    T[15] = 1.0;
}

/* ---------------------------------------------------------- FP16 rounding */

/* Round a double to the nearest IEEE binary16 value (ties to even), returned
 * as a double.  Used to model attribute storage in half precision. */
double oracle_round_half(double x) {
    if (x == 0.0 || !isfinite(x)) return x;
    double a = fabs(x);
    double spacing;
    if (a >= 65520.0) return copysign(INFINITY, x);
    if (a < 0x1p-14) {
        spacing = 0x1p-24;                    /* subnormal spacing */
    } else {
        int e;
        frexp(a, &e);                         /* a = m 2^e, m in [0.5,1) */
        spacing = ldexp(1.0, e - 1 - 10);     /* 10 fraction bits */
    }
    double q = nearbyint(a / spacing) * spacing; /* default mode: ties to even */
    return copysign(q, x);
}

/* ------------------------------------------------------ spherical harmonics */

/* Real spherical harmonics Y_k, k = l^2 + l + m, l <= 3, at unit direction d,
 * built from associated Legendre functions with the Condon-Shortley phase and
 * N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!):
 *   m > 0: sqrt2 N_lm P_l^m(cos th) cos(m ph)
 *   m < 0: sqrt2 N_l|m| P_l^|m|(cos th) sin(|m| ph)
 *   m = 0: N_l0 P_l^0(cos th). */
void oracle_sh_basis(int degree, const double d[3], double Y[16]) {
    double x = d[2];                                  /* cos(theta) */
    double st = sqrt(fmax(0.0, d[0] * d[0] + d[1] * d[1]));   /* sin(theta) */
    double ph = atan2(d[1], d[0]);
    double P[4][4] = {{0}};                           /* P[l][m] */
    for (int m = 0; m <= 3; ++m) {
        /* P_m^m = (-1)^m (2m-1)!! sin^m */
        double pmm = 1.0;
        for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * st;
        P[m][m] = pmm;
        if (m + 1 <= 3) P[m + 1][m] = x * (2.0 * m + 1.0) * pmm;
        for (int l = m + 2; l <= 3; ++l)
            P[l][m] = ((2.0 * l - 1.0) * x * P[l - 1][m] - (l + m - 1.0) * P[l - 2][m]) / (l - m);
    }
    for (int k = 0; k < 16; ++k) Y[k] = 0.0;
    for (int l = 0; l <= degree; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double f1 = 1.0, f2 = 1.0;                 /* (l-|m|)!, (l+|m|)! */
            for (int i = 2; i <= l - am; ++i) f1 *= i;
            for (int i = 2; i <= l + am; ++i) f2 *= i;
            double N = sqrt((2.0 * l + 1.0) / (4.0 * ORACLE_PI) * f1 / f2);
            double y;
            if (m > 0) y = sqrt(2.0) * N * P[l][am] * cos(am * ph);
            else if (m < 0) y = sqrt(2.0) * N * P[l][am] * sin(am * ph);
            else y = N * P[l][0];
            Y[l * l + l + m] = y;
        }
    }
}

/* ------------------------------------------------------------- preprocess */

/* Camera: az, el, tx, ty, tz, fx, fy, cx, cy (9 doubles) plus W, H. */
typedef struct {
    double R[9];      /* camera axes in world (columns) */
    double t[3];
    double fx, fy, cx, cy;
    int W, H;
} cam_t;

static void make_cam(const double* c, int W, int H, cam_t* cam) {
    oracle_camera_rotation(c[0], c[1], cam->R);
    cam->t[0] = c[2]; cam->t[1] = c[3]; cam->t[2] = c[4];
    cam->fx = c[5]; cam->fy = c[6]; cam->cx = c[7]; cam->cy = c[8];
    cam->W = W; cam->H = H;
}

static int ifloor(double x) { return (int)floor(x); }
static int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Guard bands: relative widths around each integer decision's threshold. */
typedef struct { double g_depth, g_opacity, g_radius, g_pixel; } guard_t;

/*
 * Per-Gaussian preprocess in FP64.
 *
 * Inputs: raw attributes as stored in the scene file (float32), sh_degree,
 * storage_half (1: round activated scale, quaternion, opacity and SH to
 * binary16 before use, positions stay float32), camera, guards.
 * Outputs (all length n or n*k, caller-allocated):
 *   visible[n]      1 kept, 0 culled (FP64 decision)
 *   cull[n]         0 kept, 1 near plane, 2 opacity, 3 det <= 0, 4 empty rect
 *   uvz[n*3]        projected centre (u, v) and depth z
 *   conic[n*3]      (A, B, C) of the inverse 2D covariance
 *   opac[n]         activated opacity
 *   rgb[n*3]        SH colour (clamped at 0)
 *   radius[n]       ceil(3 sqrt(lambda_max))
 *   rect[n*4]       x_lo, y_lo, x_hi, y_hi (tiles, half-open)
 *   cand[n*12]      reachable ranges within the guard band:
 *                   vis_min, vis_max, r_min, r_max, xlo_min, xlo_max,
 *                   ylo_min, ylo_max, xhi_min, xhi_max, yhi_min, yhi_max
 *   amb[n]          1 if any decision lies within its guard band
 *   dq[n*4]         decision quantities: z, opacity, 3 sqrt(lambda), lambda
 */
void oracle_preprocess(int64_t n, const float* means, const float* log_scales, const float* quats,
                       const float* opacity_logits, const float* sh, int sh_degree, int storage_half,
                       const double* camera, int W, int H, const double* guards,
                       int8_t* visible, int8_t* cull, double* uvz, double* conic, double* opac,
                       double* rgb, int32_t* radius, int32_t* rect, int32_t* cand, int8_t* amb,
                       double* dq) {
    cam_t cam;
    make_cam(camera, W, H, &cam);
    guard_t g = {guards[0], guards[1], guards[2], guards[3]};
    const int TX = (W + ORACLE_TILE - 1) / ORACLE_TILE, TY = (H + ORACLE_TILE - 1) / ORACLE_TILE;
    const double tan_fovx = W / (2.0 * cam.fx), tan_fovy = H / (2.0 * cam.fy);

    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        visible[i] = 0; cull[i] = 0; amb[i] = 0; radius[i] = 0;
        for (int k = 0; k < 3; ++k) { uvz[i * 3 + k] = 0; conic[i * 3 + k] = 0; rgb[i * 3 + k] = 0; }
        for (int k = 0; k < 4; ++k) { rect[i * 4 + k] = 0; dq[i * 4 + k] = 0; }
        for (int k = 0; k < 12; ++k) cand[i * 12 + k] = 0;
        opac[i] = 0;

        /* -- activations (Sec. 5.1) -- */
        double mu[3] = {means[i * 3], means[i * 3 + 1], means[i * 3 + 2]};
        double s[3], q[4], o;
        for (int k = 0; k < 3; ++k) s[k] = exp((double)log_scales[i * 3 + k]);
        double qn = 0;
        for (int k = 0; k < 4; ++k) qn += (double)quats[i * 4 + k] * quats[i * 4 + k];
        qn = sqrt(qn);
        for (int k = 0; k < 4; ++k) q[k] = quats[i * 4 + k] / qn;
        o = 1.0 / (1.0 + exp(-(double)opacity_logits[i]));
        double shc[16][3];
        int n_coef = (sh_degree + 1) * (sh_degree + 1);
        for (int k = 0; k < 16; ++k)
            for (int c = 0; c < 3; ++c) shc[k][c] = k < n_coef ? (double)sh[i * 48 + k * 3 + c] : 0.0;
        if (storage_half) {
            for (int k = 0; k < 3; ++k) s[k] = oracle_round_half(s[k]);
            for (int k = 0; k < 4; ++k) q[k] = oracle_round_half(q[k]);
            o = oracle_round_half(o);
            for (int k = 0; k < 16; ++k)
                for (int c = 0; c < 3; ++c) shc[k][c] = oracle_round_half(shc[k][c]);
        }

        /* -- camera transform p_c = R^T (mu - t) (Sec. 5.1 T_{w->c}) -- */
        double dw[3] = {mu[0] - cam.t[0], mu[1] - cam.t[1], mu[2] - cam.t[2]};
        double pc[3], zscale = 0;
        for (int r = 0; r < 3; ++r) {
            pc[r] = cam.R[0 * 3 + r] * dw[0] + cam.R[1 * 3 + r] * dw[1] + cam.R[2 * 3 + r] * dw[2];
        }
        for (int c = 0; c < 3; ++c) zscale += fabs(cam.R[c * 3 + 2] * dw[c]);
        double z = pc[2];
        dq[i * 4 + 0] = z;
        dq[i * 4 + 1] = o;

        /* -- near-plane and opacity culls -- */
        const double znear = 0.2, omin = 1.0 / 255.0;
        int near_amb = fabs(z - znear) <= g.g_depth * (zscale + znear);
        int op_amb = fabs(o - omin) <= g.g_opacity * omin;
        int can_keep = (z > znear || near_amb) && (o >= omin || op_amb);
        int can_cull = (z <= znear || near_amb) || (o < omin || op_amb);
        /* FP64 decision; an ambiguous cull still computes the rest so the
         * candidate ranges cover the kept outcome too */
        int keep = z > znear && o >= omin;
        if (!keep) cull[i] = z <= znear ? 1 : 2;
        if (z <= znear && !near_amb) continue;
        if (o < omin && !op_amb) continue;

        /* -- projection lambda [u v 1]^T = K p_c (Sec. 5.1) -- */
        double u = cam.fx * pc[0] / z + cam.cx;
        double v = cam.fy * pc[1] / z + cam.cy;

        /* -- 3D covariance Sigma = M M^T, M = R_q diag(s) -- */
        double w = q[0], x = q[1], y = q[2], zq = q[3];
        double Rq[9] = {1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y),
                        2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x),
                        2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)};
        double M[9], Sig[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[r * 3 + c] = Rq[r * 3 + c] * s[c];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += M[r * 3 + k] * M[c * 3 + k];
                Sig[r * 3 + c] = acc;
            }

        /* -- EWA: Sigma2 = J W Sigma W^T J^T + 0.3 I, W = R^T, J at the
         *    guard-band-clamped camera point (Zwicker et al. 2001) -- */
        double limx = 1.3 * tan_fovx, limy = 1.3 * tan_fovy;
        double txz = pc[0] / z, tyz = pc[1] / z;
        double tx = fmin(limx, fmax(-limx, txz)) * z;
        double ty = fmin(limy, fmax(-limy, tyz)) * z;
        double J[6] = {cam.fx / z, 0.0, -cam.fx * tx / (z * z),
                       0.0, cam.fy / z, -cam.fy * ty / (z * z)};
        double Wm[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Wm[r * 3 + c] = cam.R[c * 3 + r];
        double Tm[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += J[r * 3 + k] * Wm[k * 3 + c];
                Tm[r * 3 + c] = acc;
            }
        double S2[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                double acc = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc += Tm[r * 3 + a] * Sig[a * 3 + b] * Tm[c * 3 + b];
                S2[r * 2 + c] = acc;
            }
        double a2 = S2[0] + 0.3, b2 = S2[1], c2 = S2[3] + 0.3;

        /* -- conic and radius -- */
        double det = a2 * c2 - b2 * b2;
        if (det <= 0.0) { cull[i] = 3; continue; }
        double A = c2 / det, B = -b2 / det, C = a2 / det;
        double mid = 0.5 * (a2 + c2);
        double lam = mid + sqrt(fmax(0.1, mid * mid - det));
        double qr = 3.0 * sqrt(lam);
        int r = (int)ceil(qr);
        dq[i * 4 + 2] = qr;
        dq[i * 4 + 3] = lam;
        int r_min = (int)ceil(qr * (1.0 - g.g_radius)), r_max = (int)ceil(qr * (1.0 + g.g_radius));

        /* -- tile rectangle: tiles overlapped by [u-r, u+r] x [v-r, v+r] -- */
        int xlo = iclamp(ifloor((u - r) / ORACLE_TILE), 0, TX);
        int xhi = iclamp(ifloor((u + r) / ORACLE_TILE) + 1, 0, TX);
        int ylo = iclamp(ifloor((v - r) / ORACLE_TILE), 0, TY);
        int yhi = iclamp(ifloor((v + r) / ORACLE_TILE) + 1, 0, TY);
        double gu = g.g_pixel * (fabs(u - cam.cx) + fabs(cam.cx) + r_max + 1.0);
        double gv = g.g_pixel * (fabs(v - cam.cy) + fabs(cam.cy) + r_max + 1.0);
        int c_xlo_min = iclamp(ifloor((u - gu - r_max) / ORACLE_TILE), 0, TX);
        int c_xlo_max = iclamp(ifloor((u + gu - r_min) / ORACLE_TILE), 0, TX);
        int c_xhi_min = iclamp(ifloor((u - gu + r_min) / ORACLE_TILE) + 1, 0, TX);
        int c_xhi_max = iclamp(ifloor((u + gu + r_max) / ORACLE_TILE) + 1, 0, TX);
        int c_ylo_min = iclamp(ifloor((v - gv - r_max) / ORACLE_TILE), 0, TY);
        int c_ylo_max = iclamp(ifloor((v + gv - r_min) / ORACLE_TILE), 0, TY);
        int c_yhi_min = iclamp(ifloor((v - gv + r_min) / ORACLE_TILE) + 1, 0, TY);
        int c_yhi_max = iclamp(ifloor((v + gv + r_max) / ORACLE_TILE) + 1, 0, TY);

        int tiles = (xhi - xlo) * (yhi - ylo);
        int rect_can_be_empty = (c_xhi_min <= c_xlo_max) || (c_yhi_min <= c_ylo_max);
        int rect_can_be_full = (c_xhi_max > c_xlo_min) && (c_yhi_max > c_ylo_min);
        int32_t* cd = cand + i * 12;
        cd[2] = r_min; cd[3] = r_max;
        cd[4] = c_xlo_min; cd[5] = c_xlo_max; cd[6] = c_ylo_min; cd[7] = c_ylo_max;
        cd[8] = c_xhi_min; cd[9] = c_xhi_max; cd[10] = c_yhi_min; cd[11] = c_yhi_max;
        cd[0] = (can_cull || rect_can_be_empty) ? 0 : 1;
        cd[1] = (can_keep && rect_can_be_full) ? 1 : 0;
        amb[i] = (int8_t)(near_amb || op_amb || r_min != r_max || c_xlo_min != c_xlo_max ||
                          c_ylo_min != c_ylo_max || c_xhi_min != c_xhi_max || c_yhi_min != c_yhi_max);

        uvz[i * 3 + 0] = u; uvz[i * 3 + 1] = v; uvz[i * 3 + 2] = z;
        conic[i * 3 + 0] = A; conic[i * 3 + 1] = B; conic[i * 3 + 2] = C;
        opac[i] = o;
        radius[i] = r;
        rect[i * 4 + 0] = xlo; rect[i * 4 + 1] = ylo; rect[i * 4 + 2] = xhi; rect[i * 4 + 3] = yhi;
        if (!keep) continue;
        if (tiles <= 0) { cull[i] = 4; continue; }

        /* -- SH colour: direction from the camera centre to the mean -- */
        double dn = sqrt(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
        double d[3] = {dw[0] / dn, dw[1] / dn, dw[2] / dn};
        double Y[16];
        oracle_sh_basis(sh_degree, d, Y);
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < n_coef; ++k) acc += Y[k] * shc[k][c];
            rgb[i * 3 + c] = fmax(0.0, acc + 0.5);
        }
        visible[i] = 1;
    }
}

/* ------------------------------------------------------------- composite */

typedef struct { double depth; int64_t idx; } dkey_t;

static int cmp_dkey(const void* a, const void* b) {
    const dkey_t* x = (const dkey_t*)a;
    const dkey_t* y = (const dkey_t*)b;
    if (x->depth < y->depth) return -1;
    if (x->depth > y->depth) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Support rule: Gaussian i is considered at a pixel of tile (tx, ty) iff its
 * tile rectangle contains that tile. */
static inline int supports(const int32_t* rect, int64_t i, int tx, int ty) {
    const int32_t* r = rect + i * 4;
    return r[0] <= tx && tx < r[2] && r[1] <= ty && ty < r[3];
}

/* Front-to-back compositing of one pixel over an ordered list. */
static void composite_pixel(int px, int py, const dkey_t* list, int64_t len, const double* uvz,
                            const double* conic, const double* opac, const double* rgb,
                            const double bg[3], double out[4], int64_t* n_eval) {
    double T = 1.0, Cc[3] = {0, 0, 0};
    int64_t k;
    double fx = px + 0.5, fy = py + 0.5;
    for (k = 0; k < len; ++k) {
        int64_t i = list[k].idx;
        double dx = fx - uvz[i * 3 + 0], dy = fy - uvz[i * 3 + 1];
        double power = -0.5 * (conic[i * 3 + 0] * dx * dx + conic[i * 3 + 2] * dy * dy)
                       - conic[i * 3 + 1] * dx * dy;
        if (power > 0.0) continue;
        double alpha = fmin(0.99, opac[i] * exp(power));
        if (alpha < 1.0 / 255.0) continue;
        double Tn = T * (1.0 - alpha);
        if (Tn < 1e-4) { ++k; break; }
        for (int c = 0; c < 3; ++c) Cc[c] += rgb[i * 3 + c] * alpha * T;
        T = Tn;
    }
    if (n_eval) *n_eval = k;
    for (int c = 0; c < 3; ++c) out[c] = Cc[c] + T * bg[c];
    out[3] = 1.0 - T;
}

/*
 * Render pixels.  For each requested pixel: collect every visible Gaussian
 * whose tile rectangle contains the pixel's tile, order by (depth, index) and
 * composite.  All pixels of one tile have the same supported set, so it is
 * collected once per tile (same result as per pixel; a test checks this
 * against oracle_render_brute).
 *   pix: n_pix (x, y) pairs, or NULL for the whole W x H frame in row-major
 *   out: n_pix * 4 doubles (RGB + alpha); n_eval (optional): list entries
 *   visited per pixel up to and including the stopping one.
 */
void oracle_render(int64_t n, const int8_t* visible, const double* uvz, const double* conic,
                   const double* opac, const double* rgb, const int32_t* rect, int W, int H,
                   const double* bg, int64_t n_pix, const int32_t* pix, double* out, int64_t* n_eval) {
    const int TX = (W + ORACLE_TILE - 1) / ORACLE_TILE, TY = (H + ORACLE_TILE - 1) / ORACLE_TILE;
    int64_t total = pix ? n_pix : (int64_t)W * H;
    /* group requested pixels by tile */
    int64_t* tile_count = (int64_t*)calloc((size_t)TX * TY + 1, sizeof(int64_t));
    int64_t* order = (int64_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int64_t));
    for (int64_t p = 0; p < total; ++p) {
        int x = pix ? pix[p * 2] : (int)(p % W), y = pix ? pix[p * 2 + 1] : (int)(p / W);
        tile_count[(int64_t)(y / ORACLE_TILE) * TX + x / ORACLE_TILE + 1]++;
    }
    for (int64_t t = 0; t < (int64_t)TX * TY; ++t) tile_count[t + 1] += tile_count[t];
    int64_t* fill = (int64_t*)calloc((size_t)TX * TY, sizeof(int64_t));
    for (int64_t p = 0; p < total; ++p) {
        int x = pix ? pix[p * 2] : (int)(p % W), y = pix ? pix[p * 2 + 1] : (int)(p / W);
        int64_t t = (int64_t)(y / ORACLE_TILE) * TX + x / ORACLE_TILE;
        order[tile_count[t] + fill[t]++] = p;
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < (int64_t)TX * TY; ++t) {
        int64_t b = tile_count[t], e = tile_count[t + 1];
        if (b == e) continue;
        int tx = (int)(t % TX), ty = (int)(t / TX);
        int64_t cap = 1024, len = 0;
        dkey_t* list = (dkey_t*)malloc((size_t)cap * sizeof(dkey_t));
        for (int64_t i = 0; i < n; ++i) {
            if (!visible[i] || !supports(rect, i, tx, ty)) continue;
            if (len == cap) { cap *= 2; list = (dkey_t*)realloc(list, (size_t)cap * sizeof(dkey_t)); }
            list[len].depth = uvz[i * 3 + 2];
            list[len].idx = i;
            ++len;
        }
        qsort(list, (size_t)len, sizeof(dkey_t), cmp_dkey);
        for (int64_t k = b; k < e; ++k) {
            int64_t p = order[k];
            int x = pix ? pix[p * 2] : (int)(p % W), y = pix ? pix[p * 2 + 1] : (int)(p / W);
            composite_pixel(x, y, list, len, uvz, conic, opac, rgb, bg, out + p * 4,
                            n_eval ? n_eval + p : NULL);
        }
        free(list);
    }
    free(fill); free(order); free(tile_count);
}

/* Brute force: per pixel, test every Gaussian (support_rule = 1 applies the
 * tile-rectangle support; 0 lets every visible Gaussian contribute). */
void oracle_render_brute(int64_t n, const int8_t* visible, const double* uvz, const double* conic,
                         const double* opac, const double* rgb, const int32_t* rect, int W, int H,
                         const double* bg, int support_rule, double* out) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < (int64_t)W * H; ++p) {
        int x = (int)(p % W), y = (int)(p / W);
        dkey_t* list = (dkey_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(dkey_t));
        int64_t len = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!visible[i]) continue;
            if (support_rule && !supports(rect, i, x / ORACLE_TILE, y / ORACLE_TILE)) continue;
            list[len].depth = uvz[i * 3 + 2];
            list[len].idx = i;
            ++len;
        }
        qsort(list, (size_t)len, sizeof(dkey_t), cmp_dkey);
        composite_pixel(x, y, list, len, uvz, conic, opac, rgb, bg, out + p * 4, NULL);
        free(list);
    }
}

/* ------------------------------------------------------------- tile lists */

/* Number of (Gaussian, tile) pairs: sum of rectangle areas of visible ones. */
int64_t oracle_pair_count(int64_t n, const int8_t* visible, const int32_t* rect) {
    int64_t P = 0;
    for (int64_t i = 0; i < n; ++i)
        if (visible[i]) P += (int64_t)(rect[i * 4 + 2] - rect[i * 4]) * (rect[i * 4 + 3] - rect[i * 4 + 1]);
    return P;
}

/*
 * Per-tile lists for the whole frame: for each tile (row-major), the indices
 * of visible Gaussians whose rectangle contains it, ordered by (depth, index).
 *   ranges[2*T]: [start, end) of each tile in values; values[P].
 */
void oracle_tile_lists(int64_t n, const int8_t* visible, const double* uvz, const int32_t* rect,
                       int W, int H, int64_t* ranges, int32_t* values) {
    const int TX = (W + ORACLE_TILE - 1) / ORACLE_TILE, TY = (H + ORACLE_TILE - 1) / ORACLE_TILE;
    const int64_t T = (int64_t)TX * TY;
    int64_t* cnt = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        if (!visible[i]) continue;
        for (int ty = rect[i * 4 + 1]; ty < rect[i * 4 + 3]; ++ty)
            for (int tx = rect[i * 4]; tx < rect[i * 4 + 2]; ++tx) cnt[(int64_t)ty * TX + tx + 1]++;
    }
    for (int64_t t = 0; t < T; ++t) cnt[t + 1] += cnt[t];
    for (int64_t t = 0; t < T; ++t) { ranges[2 * t] = cnt[t]; ranges[2 * t + 1] = cnt[t]; }
    for (int64_t i = 0; i < n; ++i) {
        if (!visible[i]) continue;
        for (int ty = rect[i * 4 + 1]; ty < rect[i * 4 + 3]; ++ty)
            for (int tx = rect[i * 4]; tx < rect[i * 4 + 2]; ++tx) {
                int64_t t = (int64_t)ty * TX + tx;
                values[ranges[2 * t + 1]++] = (int32_t)i;
            }
    }
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < T; ++t) {
        int64_t b = ranges[2 * t], e = ranges[2 * t + 1];
        dkey_t* tmp = (dkey_t*)malloc((size_t)(e - b > 0 ? e - b : 1) * sizeof(dkey_t));
        for (int64_t k = b; k < e; ++k) { tmp[k - b].idx = values[k]; tmp[k - b].depth = uvz[values[k] * 3 + 2]; }
        qsort(tmp, (size_t)(e - b), sizeof(dkey_t), cmp_dkey);
        for (int64_t k = b; k < e; ++k) values[k] = (int32_t)tmp[k - b].idx;
        free(tmp);
    }
    free(cnt);
}

/* One tile's list (for sampled checks at full size): returns its length and
 * writes up to cap indices. */
int64_t oracle_tile_list_one(int64_t n, const int8_t* visible, const double* uvz, const int32_t* rect,
                             int tx, int ty, int64_t cap, int32_t* out) {
    int64_t len = 0;
    for (int64_t i = 0; i < n; ++i)
        if (visible[i] && supports(rect, i, tx, ty)) ++len;
    dkey_t* tmp = (dkey_t*)malloc((size_t)(len > 0 ? len : 1) * sizeof(dkey_t));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
        if (visible[i] && supports(rect, i, tx, ty)) { tmp[k].idx = i; tmp[k].depth = uvz[i * 3 + 2]; ++k; }
    qsort(tmp, (size_t)len, sizeof(dkey_t), cmp_dkey);
    for (k = 0; k < len && k < cap; ++k) out[k] = (int32_t)tmp[k].idx;
    free(tmp);
    return len;
}

/* RGBA8 encoding of a float pixel: floor(clamp(x,0,1)*255 + 0.5). */
void oracle_to_rgba8(int64_t n_pix, const double* rgba, uint8_t* out) {
    for (int64_t p = 0; p < n_pix * 4; ++p) {
        double x = fmin(1.0, fmax(0.0, rgba[p]));
        out[p] = (uint8_t)floor(x * 255.0 + 0.5);
    }
}
