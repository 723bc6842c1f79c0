/*
 * Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.
 *
 * This file holds NO rasterization arithmetic: only a counter-based random
 * number generator and the distributions that shape the synthetic scenes.
 * Both sides of every parity test read the arrays it fills; neither side's
 * arithmetic lives here.
 *
 * Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written from its published
 * definition: a 4x32-bit counter, a 2x32-bit key, ten rounds of two 32x32->64
 * multiplications with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key
 * increments 0x9E3779B9 / 0xBB67AE85.  Normals come from the Box-Muller
 * transform of pairs of uniforms.
 *
 * Every random number is addressed by (element index, block, stream, attempt)
 * so results do not depend on thread count or on chunking.
 *
 * Scene recipe (synthetic stand-in for the paper's "millions of anisotropic
 * 3D Gaussians", Sec. 1, with the attribute layout of Sec. 5.1):
 *   blob centres ~ U[-1,1]^3; isotropic blobs (sigma given) or anisotropic
 *   blobs Sigma_b = R_b diag(sigma_b^2) R_b^T with sigma_b log-uniform in
 *   [0.05, 0.4] per axis and R_b from a normalised N(0,1) quaternion;
 *   each point picks a blob uniformly, points outside [-1,1]^3 are redrawn;
 *   log-scale ~ N(-4, 0.5) per axis; raw quaternion ~ N(0,1)^4 (w,x,y,z);
 *   opacity logit ~ N(0, 1.5); SH DC ~ N(0, 0.5), bands 1..3 ~ N(0, 0.05),
 *   layout [N][16][3].
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static inline void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

/* Philox4x32-10: ctr (4 words) and key (2 words) in, 4 words out. */
void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

/* Uniform in the open interval (0,1) from one 32-bit word. */
static inline double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* Four standard normals from one Philox block (two Box-Muller pairs). */
static void normals4(uint64_t seed, uint64_t index, uint32_t block, uint32_t stream,
                     uint32_t attempt, double out[4]) {
    uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32) ^ (block << 16), stream, attempt};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    synth_philox4x32_10(ctr, key, w);
    const double two_pi = 6.283185307179586476925286766559;
    for (int p = 0; p < 2; ++p) {
        double r = sqrt(-2.0 * log(u01(w[2 * p])));
        double a = two_pi * u01(w[2 * p + 1]);
        out[2 * p] = r * cos(a);
        out[2 * p + 1] = r * sin(a);
    }
}

/* Four uniforms in (0,1) from one Philox block. */
static void uniforms4(uint64_t seed, uint64_t index, uint32_t block, uint32_t stream,
                      uint32_t attempt, double out[4]) {
    uint32_t ctr[4] = {(uint32_t)index, (uint32_t)(index >> 32) ^ (block << 16), stream, attempt};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    synth_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; ++i) out[i] = u01(w[i]);
}

/* stream ids: one per attribute so every attribute is independently addressable */
enum {
    S_BLOB_CENTRE = 1, S_BLOB_SIGMA = 2, S_BLOB_ROT = 3,
    S_PICK = 10, S_POS = 11, S_LOGSCALE = 12, S_QUAT = 13, S_OPACITY = 14,
    S_SH_DC = 15, S_SH_REST = 16,
    S_USER = 100
};

/* n normals N(0,1) for a user stream: out[i] is element i of (seed, stream). */
void synth_normals(uint64_t seed, uint32_t stream, uint64_t n, double* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < (int64_t)((n + 3) / 4); ++b) {
        double v[4];
        normals4(seed, (uint64_t)b, 0, S_USER + stream, 0, v);
        for (int j = 0; j < 4; ++j) {
            uint64_t i = (uint64_t)b * 4 + j;
            if (i < n) out[i] = v[j];
        }
    }
}

void synth_uniforms(uint64_t seed, uint32_t stream, uint64_t n, double* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < (int64_t)((n + 3) / 4); ++b) {
        double v[4];
        uniforms4(seed, (uint64_t)b, 0, S_USER + stream, 0, v);
        for (int j = 0; j < 4; ++j) {
            uint64_t i = (uint64_t)b * 4 + j;
            if (i < n) out[i] = v[j];
        }
    }
}

static void quat_to_mat(const double q_in[4], double R[9]) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/*
 * Fill a scene of n Gaussians.
 *   n_blobs, iso_sigma: isotropic blobs of std iso_sigma when iso_sigma > 0,
 *   otherwise anisotropic blobs (log-uniform per-axis std in [0.05, 0.4]).
 * Outputs (float32, caller-allocated): means[n*3], log_scales[n*3],
 * quats[n*4] (w,x,y,z, not normalised), opacity_logits[n], sh[n*48].
 * Returns the total number of rejection redraws (diagnostic).
 */
int64_t synth_scene(uint64_t seed, uint64_t n, int n_blobs, double iso_sigma,
                    float* means, float* log_scales, float* quats, float* opacity_logits,
                    float* sh) {
    if (n_blobs < 1) n_blobs = 1;
    if (n_blobs > 4096) n_blobs = 4096;
    static double centre[4096][3];
    static double L[4096][9];
    for (int b = 0; b < n_blobs; ++b) {
        double u[4];
        uniforms4(seed, (uint64_t)b, 0, S_BLOB_CENTRE, 0, u);
        for (int k = 0; k < 3; ++k) centre[b][k] = -1.0 + 2.0 * u[k];
        double sig[3];
        if (iso_sigma > 0) {
            sig[0] = sig[1] = sig[2] = iso_sigma;
            double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
            for (int k = 0; k < 9; ++k) L[b][k] = I[k] * sig[k / 3];
        } else {
            double us[4];
            uniforms4(seed, (uint64_t)b, 0, S_BLOB_SIGMA, 0, us);
            for (int k = 0; k < 3; ++k) sig[k] = exp(log(0.05) + us[k] * (log(0.4) - log(0.05)));
            double q[4], R[9];
            normals4(seed, (uint64_t)b, 0, S_BLOB_ROT, 0, q);
            quat_to_mat(q, R);
            /* L = R diag(sig): column k of R scaled by sig[k] */
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) L[b][r * 3 + c] = R[r * 3 + c] * sig[c];
        }
    }
    int64_t redraws = 0;
    #pragma omp parallel for schedule(static) reduction(+ : redraws)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        double p[3];
        for (uint32_t attempt = 0;; ++attempt) {
            double u[4], z[4];
            uniforms4(seed, (uint64_t)i, 0, S_PICK, attempt, u);
            int b = (int)(u[0] * n_blobs);
            if (b >= n_blobs) b = n_blobs - 1;
            normals4(seed, (uint64_t)i, 0, S_POS, attempt, z);
            for (int r = 0; r < 3; ++r)
                p[r] = centre[b][r] + L[b][r * 3 + 0] * z[0] + L[b][r * 3 + 1] * z[1] + L[b][r * 3 + 2] * z[2];
            if (fabs(p[0]) <= 1.0 && fabs(p[1]) <= 1.0 && fabs(p[2]) <= 1.0) break;
            ++redraws;
            if (attempt > 100000) { p[0] = p[1] = p[2] = 0.0; break; }
        }
        for (int r = 0; r < 3; ++r) means[i * 3 + r] = (float)p[r];
        double v[4];
        normals4(seed, (uint64_t)i, 0, S_LOGSCALE, 0, v);
        for (int r = 0; r < 3; ++r) log_scales[i * 3 + r] = (float)(-4.0 + 0.5 * v[r]);
        normals4(seed, (uint64_t)i, 0, S_QUAT, 0, v);
        for (int r = 0; r < 4; ++r) quats[i * 4 + r] = (float)v[r];
        normals4(seed, (uint64_t)i, 0, S_OPACITY, 0, v);
        opacity_logits[i] = (float)(1.5 * v[0]);
        normals4(seed, (uint64_t)i, 0, S_SH_DC, 0, v);
        for (int c = 0; c < 3; ++c) sh[i * 48 + c] = (float)(0.5 * v[c]);
        for (uint32_t blk = 0; blk < 12; ++blk) {   /* 45 higher-band coefficients */
            normals4(seed, (uint64_t)i, blk, S_SH_REST, 0, v);
            for (int j = 0; j < 4; ++j) {
                int k = 3 + (int)blk * 4 + j;
                if (k < 48) sh[i * 48 + k] = (float)(0.05 * v[j]);
            }
        }
    }
    return redraws;
}
