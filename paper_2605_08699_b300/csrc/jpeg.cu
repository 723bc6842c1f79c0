// Frame encoder after the blend: baseline JPEG (ITU-T T.81, sequential DCT,
// Huffman) in a JFIF file, the payload the backend returns for every pose
// request (Sec. 4.1, 5.1; the quality levels of Table 1).
//
// The encoding follows a fixed specification, so that it is reproducible
// byte for byte:
//   colour     JFIF YCbCr, weights x 65536 rounded, results clamped to 0..255
//   sampling   4:2:0, chroma = rounded mean of each 2x2 group, the image
//              extended to whole 16x16 MCUs by repeating its last column/row
//   DCT        T.81 FDCT with 13-bit fixed-point cosine weights, rows then
//              columns, one rounding shift (>> 10) between the passes
//   quantizer  Annex K.1/K.2 tables scaled by the quality (5000/q below 50,
//              200 - 2q above), nearest with halves away from zero
//   entropy    Annex K.3-K.6 Huffman tables, restart markers every
//              `restart` MCUs, 1-bit padding, 0xFF stuffing
//
// B300 mapping:
//   k_jpeg_mcu      one CTA per MCU: colour conversion, subsampling, both DCT
//                   passes and quantization in shared memory, coefficients
//                   written in zig-zag order (int16)
//   k_jpeg_entropy  one thread per restart interval (intervals are
//                   independent: predictors reset, byte-aligned), codes from
//                   shared-memory tables, bytes to a per-interval slot
//   scan            byte offsets of the intervals (device prefix scan)
//   k_jpeg_assemble one CTA per interval copies its bytes behind the header
//                   and writes the RSTn marker that follows it
#include <cmath>
#include <cstring>
#include <vector>

#include "pipeline.cuh"

namespace tigas {

namespace {

// ---------------------------------------------------------------- tables

const int kLumaBase[64] = {16, 11, 10, 16, 24,  40,  51,  61,  12, 12, 14, 19, 26,  58,  60,  55,
                           14, 13, 16, 24, 40,  57,  69,  56,  14, 17, 22, 29, 51,  87,  80,  62,
                           18, 22, 37, 56, 68,  109, 103, 77,  24, 35, 55, 64, 81,  104, 113, 92,
                           49, 64, 78, 87, 103, 121, 120, 101, 72, 92, 95, 98, 112, 100, 103, 99};
const int kChromaBase[64] = {17, 18, 24, 47, 99, 99, 99, 99, 18, 21, 26, 66, 99, 99, 99, 99,
                             24, 26, 56, 99, 99, 99, 99, 99, 47, 66, 99, 99, 99, 99, 99, 99,
                             99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99,
                             99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99};
// zig-zag position -> natural (row-major) index
const int kZz[64] = {0,  1,  8,  16, 9,  2,  3,  10, 17, 24, 32, 25, 18, 11, 4,  5,  12, 19, 26, 33, 40, 48,
                     41, 34, 27, 20, 13, 6,  7,  14, 21, 28, 35, 42, 49, 56, 57, 50, 43, 36, 29, 22, 15, 23,
                     30, 37, 44, 51, 58, 59, 52, 45, 38, 31, 39, 46, 53, 60, 61, 54, 47, 55, 62, 63};
const uint8_t kDcLBits[16] = {0, 1, 5, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0};
const uint8_t kDcCBits[16] = {0, 3, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0};
const uint8_t kDcValsT[12] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11};
const uint8_t kAcLBits[16] = {0, 2, 1, 3, 3, 2, 4, 3, 5, 5, 4, 4, 0, 0, 1, 0x7d};
const uint8_t kAcLVals[162] = {
    0x01, 0x02, 0x03, 0x00, 0x04, 0x11, 0x05, 0x12, 0x21, 0x31, 0x41, 0x06, 0x13, 0x51, 0x61, 0x07, 0x22, 0x71,
    0x14, 0x32, 0x81, 0x91, 0xa1, 0x08, 0x23, 0x42, 0xb1, 0xc1, 0x15, 0x52, 0xd1, 0xf0, 0x24, 0x33, 0x62, 0x72,
    0x82, 0x09, 0x0a, 0x16, 0x17, 0x18, 0x19, 0x1a, 0x25, 0x26, 0x27, 0x28, 0x29, 0x2a, 0x34, 0x35, 0x36, 0x37,
    0x38, 0x39, 0x3a, 0x43, 0x44, 0x45, 0x46, 0x47, 0x48, 0x49, 0x4a, 0x53, 0x54, 0x55, 0x56, 0x57, 0x58, 0x59,
    0x5a, 0x63, 0x64, 0x65, 0x66, 0x67, 0x68, 0x69, 0x6a, 0x73, 0x74, 0x75, 0x76, 0x77, 0x78, 0x79, 0x7a, 0x83,
    0x84, 0x85, 0x86, 0x87, 0x88, 0x89, 0x8a, 0x92, 0x93, 0x94, 0x95, 0x96, 0x97, 0x98, 0x99, 0x9a, 0xa2, 0xa3,
    0xa4, 0xa5, 0xa6, 0xa7, 0xa8, 0xa9, 0xaa, 0xb2, 0xb3, 0xb4, 0xb5, 0xb6, 0xb7, 0xb8, 0xb9, 0xba, 0xc2, 0xc3,
    0xc4, 0xc5, 0xc6, 0xc7, 0xc8, 0xc9, 0xca, 0xd2, 0xd3, 0xd4, 0xd5, 0xd6, 0xd7, 0xd8, 0xd9, 0xda, 0xe1, 0xe2,
    0xe3, 0xe4, 0xe5, 0xe6, 0xe7, 0xe8, 0xe9, 0xea, 0xf1, 0xf2, 0xf3, 0xf4, 0xf5, 0xf6, 0xf7, 0xf8, 0xf9, 0xfa};
const uint8_t kAcCBits[16] = {0, 2, 1, 2, 4, 4, 3, 4, 7, 5, 4, 4, 0, 1, 2, 0x77};
const uint8_t kAcCVals[162] = {
    0x00, 0x01, 0x02, 0x03, 0x11, 0x04, 0x05, 0x21, 0x31, 0x06, 0x12, 0x41, 0x51, 0x07, 0x61, 0x71, 0x13, 0x22,
    0x32, 0x81, 0x08, 0x14, 0x42, 0x91, 0xa1, 0xb1, 0xc1, 0x09, 0x23, 0x33, 0x52, 0xf0, 0x15, 0x62, 0x72, 0xd1,
    0x0a, 0x16, 0x24, 0x34, 0xe1, 0x25, 0xf1, 0x17, 0x18, 0x19, 0x1a, 0x26, 0x27, 0x28, 0x29, 0x2a, 0x35, 0x36,
    0x37, 0x38, 0x39, 0x3a, 0x43, 0x44, 0x45, 0x46, 0x47, 0x48, 0x49, 0x4a, 0x53, 0x54, 0x55, 0x56, 0x57, 0x58,
    0x59, 0x5a, 0x63, 0x64, 0x65, 0x66, 0x67, 0x68, 0x69, 0x6a, 0x73, 0x74, 0x75, 0x76, 0x77, 0x78, 0x79, 0x7a,
    0x82, 0x83, 0x84, 0x85, 0x86, 0x87, 0x88, 0x89, 0x8a, 0x92, 0x93, 0x94, 0x95, 0x96, 0x97, 0x98, 0x99, 0x9a,
    0xa2, 0xa3, 0xa4, 0xa5, 0xa6, 0xa7, 0xa8, 0xa9, 0xaa, 0xb2, 0xb3, 0xb4, 0xb5, 0xb6, 0xb7, 0xb8, 0xb9, 0xba,
    0xc2, 0xc3, 0xc4, 0xc5, 0xc6, 0xc7, 0xc8, 0xc9, 0xca, 0xd2, 0xd3, 0xd4, 0xd5, 0xd6, 0xd7, 0xd8, 0xd9, 0xda,
    0xe2, 0xe3, 0xe4, 0xe5, 0xe6, 0xe7, 0xe8, 0xe9, 0xea, 0xf2, 0xf3, 0xf4, 0xf5, 0xf6, 0xf7, 0xf8, 0xf9, 0xfa};

// Everything the kernels read, staged once per call.
struct JpegTables {
    int w[8][8];            // DCT weights, 2^13 C(u)/2 cos((2x+1)u pi/16) rounded
    int q[2][64];           // quantizer steps, natural order (0 luma, 1 chroma)
    int zz_of[64];          // natural index -> zig-zag position
    uint32_t huff[4][256];  // code | size << 16 for DC luma, AC luma, DC chroma, AC chroma
};

void canonical_codes(const uint8_t* bits, const uint8_t* vals, uint32_t* out) {
    uint32_t c = 0;
    int k = 0;
    for (int i = 0; i < 256; ++i) out[i] = 0;
    for (int len = 1; len <= 16; ++len) {
        for (int i = 0; i < bits[len - 1]; ++i) out[vals[k++]] = c++ | ((uint32_t)len << 16);
        c <<= 1;
    }
}

void make_tables(int quality, JpegTables& t) {
    for (int u = 0; u < 8; ++u)
        for (int x = 0; x < 8; ++x) {
            const double cu = u == 0 ? 1.0 / std::sqrt(2.0) : 1.0;
            t.w[u][x] = (int)std::floor(8192.0 * 0.5 * cu * std::cos((2.0 * x + 1.0) * u * M_PI / 16.0) + 0.5);
        }
    const int qq = quality < 1 ? 1 : (quality > 100 ? 100 : quality);
    const int scale = qq < 50 ? 5000 / qq : 200 - 2 * qq;
    for (int i = 0; i < 64; ++i) {
        const int l = (kLumaBase[i] * scale + 50) / 100, c = (kChromaBase[i] * scale + 50) / 100;
        t.q[0][i] = l < 1 ? 1 : (l > 255 ? 255 : l);
        t.q[1][i] = c < 1 ? 1 : (c > 255 ? 255 : c);
    }
    for (int k = 0; k < 64; ++k) t.zz_of[kZz[k]] = k;
    canonical_codes(kDcLBits, kDcValsT, t.huff[0]);
    canonical_codes(kAcLBits, kAcLVals, t.huff[1]);
    canonical_codes(kDcCBits, kDcValsT, t.huff[2]);
    canonical_codes(kAcCBits, kAcCVals, t.huff[3]);
}

void put16(std::vector<uint8_t>& v, int x) {
    v.push_back((uint8_t)(x >> 8));
    v.push_back((uint8_t)x);
}
void put_dht(std::vector<uint8_t>& v, int cls_id, const uint8_t* bits, const uint8_t* vals, int n) {
    put16(v, 0xFFC4);
    put16(v, 19 + n);
    v.push_back((uint8_t)cls_id);
    v.insert(v.end(), bits, bits + 16);
    v.insert(v.end(), vals, vals + n);
}

// SOI .. SOS of the file
std::vector<uint8_t> make_header(int w, int h, int restart, const JpegTables& t) {
    std::vector<uint8_t> v;
    put16(v, 0xFFD8);
    put16(v, 0xFFE0);
    put16(v, 16);
    const uint8_t jfif[14] = {'J', 'F', 'I', 'F', 0, 1, 1, 0, 0, 1, 0, 1, 0, 0};
    v.insert(v.end(), jfif, jfif + 14);
    for (int tq = 0; tq < 2; ++tq) {
        put16(v, 0xFFDB);
        put16(v, 67);
        v.push_back((uint8_t)tq);
        for (int k = 0; k < 64; ++k) v.push_back((uint8_t)t.q[tq][kZz[k]]);
    }
    put16(v, 0xFFC0);
    put16(v, 17);
    v.push_back(8);
    put16(v, h);
    put16(v, w);
    v.push_back(3);
    const uint8_t comps[9] = {1, 0x22, 0, 2, 0x11, 1, 3, 0x11, 1};
    v.insert(v.end(), comps, comps + 9);
    put_dht(v, 0x00, kDcLBits, kDcValsT, 12);
    put_dht(v, 0x10, kAcLBits, kAcLVals, 162);
    put_dht(v, 0x01, kDcCBits, kDcValsT, 12);
    put_dht(v, 0x11, kAcCBits, kAcCVals, 162);
    put16(v, 0xFFDD);
    put16(v, 4);
    put16(v, restart);
    put16(v, 0xFFDA);
    put16(v, 12);
    v.push_back(3);
    const uint8_t sos[6] = {1, 0x00, 2, 0x11, 3, 0x11};
    v.insert(v.end(), sos, sos + 6);
    v.push_back(0);
    v.push_back(63);
    v.push_back(0);
    return v;
}

// ------------------------------------------------------------- kernels

__device__ inline void rgb_to_ycc(int r, int g, int b, int& y, int& cb, int& cr) {
    y = min(255, (19595 * r + 38470 * g + 7471 * b + 32768) >> 16);
    cb = min(255, (-11058 * r - 21710 * g + 32768 * b + (128 << 16) + 32768) >> 16);
    cr = min(255, (32768 * r - 27439 * g - 5329 * b + (128 << 16) + 32768) >> 16);
}

__device__ inline int quantize(int32_t c, int q) {
    const int64_t den = (int64_t)q << 16;
    const int64_t a = c < 0 ? -(int64_t)c : (int64_t)c;
    const int64_t m = (a + (den >> 1)) / den;
    return (int)(c < 0 ? -m : m);
}

// One MCU per CTA (256 threads): coefficients of its 6 blocks (Y00 Y01 Y10 Y11 Cb Cr)
// in zig-zag order at coef[(mcu * 6 + b) * 64].
__global__ void __launch_bounds__(256)
k_jpeg_mcu(const uint8_t* __restrict__ rgba, int W, int H, int mw, const JpegTables* __restrict__ tab,
           int16_t* __restrict__ coef) {
    __shared__ int s_y[256], s_cb[256], s_cr[256];
    __shared__ int s_s[6][64];
    __shared__ int32_t s_r[6][64];
    __shared__ int s_w[8][8];
    __shared__ int s_q[2][64];
    __shared__ int s_zz[64];
    const int t = threadIdx.x;
    if (t < 64) {
        s_w[t >> 3][t & 7] = tab->w[t >> 3][t & 7];
        s_q[0][t] = tab->q[0][t];
        s_q[1][t] = tab->q[1][t];
        s_zz[t] = tab->zz_of[t];
    }
    const int mcu = blockIdx.x, mx = mcu % mw, my = mcu / mw;
    {
        const int x = min(mx * 16 + (t & 15), W - 1), y = min(my * 16 + (t >> 4), H - 1);
        const uchar4 p = reinterpret_cast<const uchar4*>(rgba)[(size_t)y * W + x];
        int Y, Cb, Cr;
        rgb_to_ycc(p.x, p.y, p.z, Y, Cb, Cr);
        s_y[t] = Y;
        s_cb[t] = Cb;
        s_cr[t] = Cr;
    }
    __syncthreads();
    {   // level-shifted samples of the 6 blocks
        const int b = t >> 6, i = t & 63, yy = i >> 3, xx = i & 7;   // b in 0..3: Y quadrants
        s_s[b][i] = s_y[((b >> 1) * 8 + yy) * 16 + (b & 1) * 8 + xx] - 128;
        if (t < 128) {
            const int c = t >> 6;
            const int* src = c ? s_cr : s_cb;
            const int sum = src[(2 * yy) * 16 + 2 * xx] + src[(2 * yy) * 16 + 2 * xx + 1] +
                            src[(2 * yy + 1) * 16 + 2 * xx] + src[(2 * yy + 1) * 16 + 2 * xx + 1];
            s_s[4 + c][i] = ((sum + 2) >> 2) - 128;
        }
    }
    __syncthreads();
    for (int it = t; it < 384; it += 256) {   // rows: r[b][y][u] = sum_x w[u][x] s[b][y][x]
        const int b = it >> 6, y = (it >> 3) & 7, u = it & 7;
        int32_t acc = 0;
#pragma unroll
        for (int x = 0; x < 8; ++x) acc += s_w[u][x] * s_s[b][y * 8 + x];
        s_r[b][y * 8 + u] = (acc + 512) >> 10;
    }
    __syncthreads();
    for (int it = t; it < 384; it += 256) {   // columns, quantization, zig-zag store
        const int b = it >> 6, v = (it >> 3) & 7, u = it & 7;
        int32_t acc = 0;
#pragma unroll
        for (int y = 0; y < 8; ++y) acc += s_w[v][y] * s_r[b][y * 8 + u];
        const int nat = v * 8 + u;
        coef[((size_t)mcu * 6 + b) * 64 + s_zz[nat]] = (int16_t)quantize(acc, s_q[b < 4 ? 0 : 1][nat]);
    }
}

struct BitOut {
    uint8_t* p;
    uint32_t n, cap;
    uint64_t acc;
    int nbits;
    bool over;
    __device__ inline void byte(uint8_t b) {
        if (n < cap) p[n] = b; else over = true;
        ++n;
    }
    __device__ inline void bits(uint32_t v, int k) {
        if (k == 0) return;
        acc = (acc << k) | (v & ((1u << k) - 1u));
        nbits += k;
        while (nbits >= 8) {
            const uint8_t b = (uint8_t)(acc >> (nbits - 8));
            byte(b);
            if (b == 0xFF) byte(0x00);
            nbits -= 8;
        }
    }
    __device__ inline void flush() {
        if (nbits > 0) bits(0x7F, 8 - nbits);
    }
};

__device__ inline int category(int v) { return v == 0 ? 0 : 32 - __clz(v < 0 ? -v : v); }

// One thread per restart interval: its MCUs' entropy-coded bytes at slot i.
__global__ void __launch_bounds__(128)
k_jpeg_entropy(const int16_t* __restrict__ coef, int n_mcu, int restart, int n_int, const JpegTables* __restrict__ tab,
               uint8_t* __restrict__ slots, uint32_t slot_bytes, uint32_t* __restrict__ lens, uint32_t* __restrict__ flags) {
    __shared__ uint32_t s_h[4][256];
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) (&s_h[0][0])[k] = (&tab->huff[0][0])[k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    BitOut o{slots + (size_t)i * slot_bytes, 0, slot_bytes, 0, 0, false};
    int pred[3] = {0, 0, 0};
    const int m0 = i * restart, m1 = min(n_mcu, m0 + restart);
    for (int m = m0; m < m1; ++m)
        for (int b = 0; b < 6; ++b) {
            const int16_t* z = coef + ((size_t)m * 6 + b) * 64;
            const int comp = b < 4 ? 0 : b - 3;
            const uint32_t* dc = s_h[comp ? 2 : 0];
            const uint32_t* ac = s_h[comp ? 3 : 1];
            const int diff = z[0] - pred[comp];
            pred[comp] = z[0];
            int n = category(diff);
            o.bits(dc[n] & 0xFFFFu, (int)(dc[n] >> 16));
            if (n) o.bits((uint32_t)(diff < 0 ? diff - 1 : diff), n);
            int run = 0;
            for (int k = 1; k < 64; ++k) {
                const int v = z[k];
                if (v == 0) {
                    ++run;
                    continue;
                }
                while (run > 15) {
                    o.bits(ac[0xF0] & 0xFFFFu, (int)(ac[0xF0] >> 16));
                    run -= 16;
                }
                n = category(v);
                const int sym = (run << 4) | n;
                o.bits(ac[sym] & 0xFFFFu, (int)(ac[sym] >> 16));
                o.bits((uint32_t)(v < 0 ? v - 1 : v), n);
                run = 0;
            }
            if (run > 0) o.bits(ac[0x00] & 0xFFFFu, (int)(ac[0x00] >> 16));
        }
    o.flush();
    lens[i] = o.n + (i + 1 < n_int ? 2u : 0u);   // an RSTn marker follows every interval but the last
    if (o.over) atomicOr(flags, 1u);
}

// One warp per restart interval (intervals of at most kWarpMaxMcu MCUs): the
// same bytes as k_jpeg_entropy.  Per block, lane l takes zig-zag coefficients
// 2l and 2l + 1; a warp max-scan finds each nonzero coefficient's preceding
// nonzero (its zero run) and a warp sum-scan its bit offset; every lane ORs
// its codes into the warp's bit buffer in shared memory.  The finished bit
// string is padded with 1-bits to a byte and copied out with a 0x00 after
// every 0xFF byte (positions from a ballot prefix count).
constexpr int kWarpMaxMcu = 4;
constexpr int kBlockMaxBits = 11 + 11 + 63 * (16 + 10);            // DC code + bits, 63 x (AC code + bits)
constexpr int kWarpBufWords = (kWarpMaxMcu * 6 * kBlockMaxBits + 8 + 31) / 32;
constexpr int kEntropyWarps = 4;

__device__ inline void put_bits(uint32_t* buf, uint32_t pos, uint32_t v, int len) {   // len 1..32, MSB first
    if (len <= 0) return;
    v &= len == 32 ? 0xFFFFFFFFu : ((1u << len) - 1u);
    const uint32_t w = pos >> 5, off = pos & 31u;
    if (off + (uint32_t)len <= 32u) {
        atomicOr(&buf[w], v << (32u - off - (uint32_t)len));
    } else {
        const uint32_t hi = 32u - off, lo = (uint32_t)len - hi;
        atomicOr(&buf[w], v >> lo);
        atomicOr(&buf[w + 1], v << (32u - lo));
    }
}

__global__ void __launch_bounds__(32 * kEntropyWarps)
k_jpeg_entropy_warp(const int16_t* __restrict__ coef, int n_mcu, int restart, int n_int,
                    const JpegTables* __restrict__ tab, uint8_t* __restrict__ slots, uint32_t slot_bytes,
                    uint32_t* __restrict__ lens, uint32_t* __restrict__ flags) {
    __shared__ uint32_t s_h[4][256];
    __shared__ uint32_t s_buf[kEntropyWarps][kWarpBufWords];
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) (&s_h[0][0])[k] = (&tab->huff[0][0])[k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* buf = s_buf[warp];
    for (int k = lane; k < kWarpBufWords; k += 32) buf[k] = 0u;
    __syncthreads();
    const int i = blockIdx.x * kEntropyWarps + warp;
    if (i >= n_int) return;   // warp-uniform
    const uint32_t full = 0xFFFFFFFFu;
    int pred[3] = {0, 0, 0};
    uint32_t bitpos = 0;
    const int m0 = i * restart, m1 = min(n_mcu, m0 + restart);
    for (int m = m0; m < m1; ++m)
        for (int b = 0; b < 6; ++b) {
            const int32_t word = reinterpret_cast<const int32_t*>(coef + ((size_t)m * 6 + b) * 64)[lane];
            const int lo = (int16_t)(word & 0xFFFF), hi = (int16_t)((uint32_t)word >> 16);
            const int comp = b < 4 ? 0 : b - 3;
            const uint32_t* dc = s_h[comp ? 2 : 0];
            const uint32_t* ac = s_h[comp ? 3 : 1];
            const int z0 = __shfl_sync(full, lo, 0);
            const int diff = z0 - pred[comp];
            pred[comp] = z0;
            // the lane's items: [DC (lane 0)] then AC positions 2 lane (lane > 0) and 2 lane + 1
            const int p_lo = 2 * lane, p_hi = 2 * lane + 1;
            const bool nz_lo = lane > 0 && lo != 0, nz_hi = hi != 0;
            // position of the last nonzero AC coefficient at or below this lane's positions
            int last = nz_hi ? p_hi : (nz_lo ? p_lo : 0);
            int incl = last;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(full, incl, d);
                if (lane >= d) incl = max(incl, y);
            }
            const int before = __shfl_up_sync(full, incl, 1);
            const int prev_lane = lane > 0 ? before : 0;   // last nonzero AC position before this lane
            const int last_nz = __shfl_sync(full, incl, 31);
            const uint32_t zrl = ac[0xF0];
            const int zrl_len = (int)(zrl >> 16);
            // bit lengths of the lane's items
            int n_dc = 0, len_dc = 0;
            if (lane == 0) {
                n_dc = category(diff);
                len_dc = (int)(dc[n_dc] >> 16) + n_dc;
            }
            int run_lo = 0, n_lo = 0, len_lo = 0, run_hi = 0, n_hi = 0, len_hi = 0;
            if (nz_lo) {
                run_lo = p_lo - prev_lane - 1;
                n_lo = category(lo);
                len_lo = (run_lo >> 4) * zrl_len + (int)(ac[((run_lo & 15) << 4) | n_lo] >> 16) + n_lo;
            }
            if (nz_hi) {
                run_hi = p_hi - (nz_lo ? p_lo : prev_lane) - 1;
                n_hi = category(hi);
                len_hi = (run_hi >> 4) * zrl_len + (int)(ac[((run_hi & 15) << 4) | n_hi] >> 16) + n_hi;
            }
            const int mine = len_dc + len_lo + len_hi;
            int sum = mine;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(full, sum, d);
                if (lane >= d) sum += y;
            }
            const int total = __shfl_sync(full, sum, 31);
            uint32_t pos = bitpos + (uint32_t)(sum - mine);
            if (lane == 0) {
                const uint32_t c = dc[n_dc];
                put_bits(buf, pos, c & 0xFFFFu, (int)(c >> 16));
                pos += c >> 16;
                put_bits(buf, pos, (uint32_t)(diff < 0 ? diff - 1 : diff), n_dc);
                pos += (uint32_t)n_dc;
            }
            auto put_ac = [&](int run, int n, int v) {
                for (int z = 0; z < (run >> 4); ++z) {
                    put_bits(buf, pos, zrl & 0xFFFFu, zrl_len);
                    pos += (uint32_t)zrl_len;
                }
                const uint32_t c = ac[((run & 15) << 4) | n];
                put_bits(buf, pos, c & 0xFFFFu, (int)(c >> 16));
                pos += c >> 16;
                put_bits(buf, pos, (uint32_t)(v < 0 ? v - 1 : v), n);
                pos += (uint32_t)n;
            };
            if (nz_lo) put_ac(run_lo, n_lo, lo);
            if (nz_hi) put_ac(run_hi, n_hi, hi);
            bitpos += (uint32_t)total;
            if (last_nz < 63) {   // end of block after the last nonzero coefficient
                const uint32_t eob = ac[0x00];
                if (lane == 0) put_bits(buf, bitpos, eob & 0xFFFFu, (int)(eob >> 16));
                bitpos += eob >> 16;
            }
        }
    const uint32_t pad = (8u - (bitpos & 7u)) & 7u;
    if (lane == 0 && pad) put_bits(buf, bitpos, 0xFFu, (int)pad);
    __syncwarp();
    const uint32_t n_bytes = (bitpos + pad) >> 3;
    uint8_t* out = slots + (size_t)i * slot_bytes;
    uint32_t stuffed = 0;   // 0x00 bytes inserted so far
    bool over = false;
    for (uint32_t j0 = 0; j0 < n_bytes; j0 += 32) {
        const uint32_t j = j0 + (uint32_t)lane;
        uint32_t byte = 0;
        if (j < n_bytes) byte = (buf[j >> 2] >> (24u - 8u * (j & 3u))) & 0xFFu;
        const bool ff = j < n_bytes && byte == 0xFFu;
        const uint32_t m = __ballot_sync(full, ff);
        if (j < n_bytes) {
            const uint32_t o = j + stuffed + (uint32_t)__popc(m & ((1u << lane) - 1u));
            if (o < slot_bytes) out[o] = (uint8_t)byte; else over = true;
            if (ff) {
                if (o + 1 < slot_bytes) out[o + 1] = 0x00; else over = true;
            }
        }
        stuffed += (uint32_t)__popc(m);
    }
    if (__any_sync(full, over) && lane == 0) atomicOr(flags, 1u);
    if (lane == 0) lens[i] = n_bytes + stuffed + (i + 1 < n_int ? 2u : 0u);
}

// One CTA per interval: its bytes (and the RSTn marker after it) at out[offsets[i]].
__global__ void __launch_bounds__(256)
k_jpeg_assemble(const uint8_t* __restrict__ slots, uint32_t slot_bytes, const uint32_t* __restrict__ lens,
                const uint32_t* __restrict__ offsets, int n_int, uint8_t* __restrict__ out, uint64_t out_cap,
                uint32_t* __restrict__ flags) {
    const int i = blockIdx.x;
    const uint64_t off = offsets[i];
    const uint32_t len = lens[i];
    uint32_t data = len - (i + 1 < n_int ? 2u : 0u);
    if (data > slot_bytes) data = slot_bytes;   // cannot happen (the slot is a worst case; the host reports it)
    if (off + len > out_cap) {
        if (threadIdx.x == 0) atomicOr(flags, 2u);
        return;
    }
    const uint8_t* src = slots + (size_t)i * slot_bytes;
    for (uint32_t k = threadIdx.x; k < data; k += blockDim.x) out[off + k] = src[k];
    if (threadIdx.x == 0 && i + 1 < n_int) {
        out[off + data] = 0xFF;
        out[off + data + 1] = (uint8_t)(0xD0 + (i & 7));
    }
}

}  // namespace

Status jpeg_encode(RenderContext& ctx, const uint8_t* rgba, int W, int H, int quality, int restart, uint8_t* out,
                   uint64_t cap, uint64_t* out_len, cudaStream_t st) {
    if (W < 1 || H < 1 || W > 65535 || H > 65535) return {TIGAS_ERR_INVALID, "jpeg: width/height out of 1..65535"};
    if (quality < 1 || quality > 100) return {TIGAS_ERR_INVALID, "jpeg: quality out of 1..100"};
    if (restart < 1 || restart > 65535) return {TIGAS_ERR_INVALID, "jpeg: restart interval out of 1..65535 MCUs"};
    if (!rgba || !out_len) return {TIGAS_ERR_INVALID, "jpeg: null argument"};
    JpegTables tab;
    make_tables(quality, tab);
    const std::vector<uint8_t> hdr = make_header(W, H, restart, tab);
    const int mw = (W + 15) / 16, mh = (H + 15) / 16, n_mcu = mw * mh;
    const int n_int = (n_mcu + restart - 1) / restart;
    // worst case per block: 16 + 11 bits of DC, 63 x (16 + 10) bits of AC, every byte stuffed
    const uint64_t slot64 = (uint64_t)restart * 6 * ((16 + 11 + 63 * 26 + 7) / 8) * 2 + 16;
    if (slot64 > 0xFFFFFFFFull) return {TIGAS_ERR_INVALID, "jpeg: restart interval too long"};
    const uint32_t slot = (uint32_t)((slot64 + 15) & ~15ull);
    const bool dev_in = is_device_pointer(rgba), dev_out = is_device_pointer(out);
    const uint64_t entropy_cap = (uint64_t)n_int * slot;
    const uint64_t stream_cap = entropy_cap + 2ull * n_int;   // bytes plus the RSTn markers
    const size_t px = (size_t)W * H * 4;
    const size_t bytes = sizeof(JpegTables) + (size_t)n_mcu * 6 * 64 * 2 + entropy_cap + (size_t)(n_int + 1) * 8 +
                         scan_tmp_words((uint64_t)n_int + 1) * 4 + (dev_in ? 0 : px) + (dev_out ? 0 : stream_cap) +
                         64 + 16 * 256;
    TIGAS_TRY(ctx.jpeg.reserve(bytes));
    ctx.jpeg.reset();
    JpegTables* d_tab = ctx.jpeg.take<JpegTables>(1);
    int16_t* d_coef = ctx.jpeg.take<int16_t>((size_t)n_mcu * 6 * 64);
    uint8_t* d_slots = ctx.jpeg.take<uint8_t>(entropy_cap);
    uint32_t* d_lens = ctx.jpeg.take<uint32_t>(n_int + 1);
    uint32_t* d_offs = ctx.jpeg.take<uint32_t>(n_int + 1);
    uint32_t* d_tmp = ctx.jpeg.take<uint32_t>(scan_tmp_words((uint64_t)n_int + 1));
    uint32_t* d_flags = ctx.jpeg.take<uint32_t>(2);
    uint64_t* d_total = ctx.jpeg.take<uint64_t>(1);
    const uint8_t* d_in = rgba;
    if (!dev_in) {
        uint8_t* stage = ctx.jpeg.take<uint8_t>(px);
        d_in = stage;
        if (ctx.jpeg.over) return {TIGAS_ERR_CUDA, "jpeg workspace layout exceeds its reservation"};
        TIGAS_CUDA_TRY(cudaMemcpyAsync(stage, rgba, px, cudaMemcpyHostToDevice, st));
    }
    uint8_t* d_ent = dev_out ? nullptr : ctx.jpeg.take<uint8_t>(stream_cap);
    if (ctx.jpeg.over) return {TIGAS_ERR_CUDA, "jpeg workspace layout exceeds its reservation"};
    TIGAS_CUDA_TRY(cudaMemcpyAsync(d_tab, &tab, sizeof(JpegTables), cudaMemcpyHostToDevice, st));
    TIGAS_CUDA_TRY(cudaMemsetAsync(d_flags, 0, 8, st));
    TIGAS_CUDA_TRY(cudaMemsetAsync(d_lens + n_int, 0, 4, st));   // the scan's extra zero
    k_jpeg_mcu<<<n_mcu, 256, 0, st>>>(d_in, W, H, mw, d_tab, d_coef);
    TIGAS_LAUNCHED();
    if (restart <= kWarpMaxMcu)
        k_jpeg_entropy_warp<<<(n_int + kEntropyWarps - 1) / kEntropyWarps, 32 * kEntropyWarps, 0, st>>>(
            d_coef, n_mcu, restart, n_int, d_tab, d_slots, slot, d_lens, d_flags);
    else
        k_jpeg_entropy<<<(n_int + 31) / 32, 32, 0, st>>>(d_coef, n_mcu, restart, n_int, d_tab, d_slots, slot, d_lens,
                                                        d_flags);
    TIGAS_LAUNCHED();
    TIGAS_TRY(launch_scan_u32(d_lens, nullptr, d_offs, (uint64_t)n_int + 1, d_total, d_tmp, st));
    // entropy-coded data: straight into the caller's device buffer behind the header, or staged
    uint8_t* dst = dev_out ? out + hdr.size() : d_ent;
    const uint64_t dst_cap = dev_out ? (cap > hdr.size() + 2 ? cap - hdr.size() - 2 : 0) : stream_cap;
    k_jpeg_assemble<<<n_int, 256, 0, st>>>(d_slots, slot, d_lens, d_offs, n_int, dst, dst_cap, d_flags);
    TIGAS_LAUNCHED();
    uint64_t total = 0;
    uint32_t flags[2] = {0, 0};
    TIGAS_CUDA_TRY(cudaMemcpyAsync(&total, d_total, 8, cudaMemcpyDeviceToHost, st));
    TIGAS_CUDA_TRY(cudaMemcpyAsync(flags, d_flags, 8, cudaMemcpyDeviceToHost, st));
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    if (flags[0] & 1u) return {TIGAS_ERR_CUDA, "jpeg: an interval outgrew its worst-case slot"};
    const uint64_t need = hdr.size() + total + 2;
    *out_len = need;
    if (need > cap || (flags[0] & 2u)) return {TIGAS_ERR_OVERFLOW, "jpeg: output buffer too small"};
    const uint8_t eoi[2] = {0xFF, 0xD9};
    if (dev_out) {
        TIGAS_CUDA_TRY(cudaMemcpyAsync(out, hdr.data(), hdr.size(), cudaMemcpyHostToDevice, st));
        TIGAS_CUDA_TRY(cudaMemcpyAsync(out + hdr.size() + total, eoi, 2, cudaMemcpyHostToDevice, st));
    } else {
        std::memcpy(out, hdr.data(), hdr.size());
        TIGAS_CUDA_TRY(cudaMemcpyAsync(out + hdr.size(), d_ent, total, cudaMemcpyDeviceToHost, st));
        std::memcpy(out + hdr.size() + total, eoi, 2);
    }
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    return {};
}

}  // namespace tigas
