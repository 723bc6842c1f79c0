/* CPU oracle of the frame encoder that follows the blend: baseline JPEG
 * (ITU-T T.81, sequential DCT, Huffman) in a JFIF file, the response payload
 * of every render request (Sec. 4.1, 5.1; quality levels of Table 1).
 *
 * Test infrastructure only: the tests, smoke() and bench.py's CPU leg load it;
 * it shares no code with the CUDA encoder.
 *
 * The encoding is fully specified here so that the CUDA encoder can be held
 * to it byte for byte:
 *   colour      JFIF YCbCr with 16-bit fixed-point weights (the JFIF
 *               formulas times 65536, rounded), results clamped to 0..255
 *   sampling    4:2:0; chroma = rounded mean of each 2x2 group; the image is
 *               extended to whole 16x16 MCUs by repeating its last column/row
 *   DCT         the T.81 FDCT definition with 13-bit fixed-point cosine
 *               weights, rows then columns, one rounding shift between them
 *   quantizer   T.81 Annex K.1/K.2 tables scaled by the quality (reading: the
 *               Independent JPEG Group's convention, 5000/q below 50 and
 *               200 - 2q above), the coefficient rounded to nearest, halves
 *               away from zero
 *   entropy     Annex K.3-K.6 Huffman tables, DC differences per component,
 *               AC run/size symbols with ZRL and EOB, restart markers every
 *               `restart` MCUs (predictors reset, bit buffer padded with 1s),
 *               0xFF followed by a stuffed 0x00
 * The fixed-point DCT is pinned against the double-precision definition, the
 * bitstream by an independent decoder in the tests. */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- tables */

/* Table K.1 (luminance) and K.2 (chrominance), natural (row-major) order. */
static const int kBaseLuma[64] = {
    16, 11, 10, 16, 24,  40,  51,  61,  12, 12, 14, 19, 26,  58,  60,  55,
    14, 13, 16, 24, 40,  57,  69,  56,  14, 17, 22, 29, 51,  87,  80,  62,
    18, 22, 37, 56, 68,  109, 103, 77,  24, 35, 55, 64, 81,  104, 113, 92,
    49, 64, 78, 87, 103, 121, 120, 101, 72, 92, 95, 98, 112, 100, 103, 99};
static const int kBaseChroma[64] = {
    17, 18, 24, 47, 99, 99, 99, 99, 18, 21, 26, 66, 99, 99, 99, 99,
    24, 26, 56, 99, 99, 99, 99, 99, 47, 66, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99,
    99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99, 99};

/* zig-zag position k -> natural index (Figure A.6) */
static const int kZigzag[64] = {
    0,  1,  8,  16, 9,  2,  3,  10, 17, 24, 32, 25, 18, 11, 4,  5,
    12, 19, 26, 33, 40, 48, 41, 34, 27, 20, 13, 6,  7,  14, 21, 28,
    35, 42, 49, 56, 57, 50, 43, 36, 29, 22, 15, 23, 30, 37, 44, 51,
    58, 59, 52, 45, 38, 31, 39, 46, 53, 60, 61, 54, 47, 55, 62, 63};

/* Huffman tables K.3-K.6: number of codes of each length 1..16, then values. */
static const uint8_t kDcLumaBits[16] = {0, 1, 5, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0};
static const uint8_t kDcChromaBits[16] = {0, 3, 1, 1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0};
static const uint8_t kDcVals[12] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11};
static const uint8_t kAcLumaBits[16] = {0, 2, 1, 3, 3, 2, 4, 3, 5, 5, 4, 4, 0, 0, 1, 0x7d};
static const uint8_t kAcLumaVals[162] = {
    0x01, 0x02, 0x03, 0x00, 0x04, 0x11, 0x05, 0x12, 0x21, 0x31, 0x41, 0x06, 0x13, 0x51, 0x61, 0x07, 0x22, 0x71,
    0x14, 0x32, 0x81, 0x91, 0xa1, 0x08, 0x23, 0x42, 0xb1, 0xc1, 0x15, 0x52, 0xd1, 0xf0, 0x24, 0x33, 0x62, 0x72,
    0x82, 0x09, 0x0a, 0x16, 0x17, 0x18, 0x19, 0x1a, 0x25, 0x26, 0x27, 0x28, 0x29, 0x2a, 0x34, 0x35, 0x36, 0x37,
    0x38, 0x39, 0x3a, 0x43, 0x44, 0x45, 0x46, 0x47, 0x48, 0x49, 0x4a, 0x53, 0x54, 0x55, 0x56, 0x57, 0x58, 0x59,
    0x5a, 0x63, 0x64, 0x65, 0x66, 0x67, 0x68, 0x69, 0x6a, 0x73, 0x74, 0x75, 0x76, 0x77, 0x78, 0x79, 0x7a, 0x83,
    0x84, 0x85, 0x86, 0x87, 0x88, 0x89, 0x8a, 0x92, 0x93, 0x94, 0x95, 0x96, 0x97, 0x98, 0x99, 0x9a, 0xa2, 0xa3,
    0xa4, 0xa5, 0xa6, 0xa7, 0xa8, 0xa9, 0xaa, 0xb2, 0xb3, 0xb4, 0xb5, 0xb6, 0xb7, 0xb8, 0xb9, 0xba, 0xc2, 0xc3,
    0xc4, 0xc5, 0xc6, 0xc7, 0xc8, 0xc9, 0xca, 0xd2, 0xd3, 0xd4, 0xd5, 0xd6, 0xd7, 0xd8, 0xd9, 0xda, 0xe1, 0xe2,
    0xe3, 0xe4, 0xe5, 0xe6, 0xe7, 0xe8, 0xe9, 0xea, 0xf1, 0xf2, 0xf3, 0xf4, 0xf5, 0xf6, 0xf7, 0xf8, 0xf9, 0xfa};
static const uint8_t kAcChromaBits[16] = {0, 2, 1, 2, 4, 4, 3, 4, 7, 5, 4, 4, 0, 1, 2, 0x77};
static const uint8_t kAcChromaVals[162] = {
    0x00, 0x01, 0x02, 0x03, 0x11, 0x04, 0x05, 0x21, 0x31, 0x06, 0x12, 0x41, 0x51, 0x07, 0x61, 0x71, 0x13, 0x22,
    0x32, 0x81, 0x08, 0x14, 0x42, 0x91, 0xa1, 0xb1, 0xc1, 0x09, 0x23, 0x33, 0x52, 0xf0, 0x15, 0x62, 0x72, 0xd1,
    0x0a, 0x16, 0x24, 0x34, 0xe1, 0x25, 0xf1, 0x17, 0x18, 0x19, 0x1a, 0x26, 0x27, 0x28, 0x29, 0x2a, 0x35, 0x36,
    0x37, 0x38, 0x39, 0x3a, 0x43, 0x44, 0x45, 0x46, 0x47, 0x48, 0x49, 0x4a, 0x53, 0x54, 0x55, 0x56, 0x57, 0x58,
    0x59, 0x5a, 0x63, 0x64, 0x65, 0x66, 0x67, 0x68, 0x69, 0x6a, 0x73, 0x74, 0x75, 0x76, 0x77, 0x78, 0x79, 0x7a,
    0x82, 0x83, 0x84, 0x85, 0x86, 0x87, 0x88, 0x89, 0x8a, 0x92, 0x93, 0x94, 0x95, 0x96, 0x97, 0x98, 0x99, 0x9a,
    0xa2, 0xa3, 0xa4, 0xa5, 0xa6, 0xa7, 0xa8, 0xa9, 0xaa, 0xb2, 0xb3, 0xb4, 0xb5, 0xb6, 0xb7, 0xb8, 0xb9, 0xba,
    0xc2, 0xc3, 0xc4, 0xc5, 0xc6, 0xc7, 0xc8, 0xc9, 0xca, 0xd2, 0xd3, 0xd4, 0xd5, 0xd6, 0xd7, 0xd8, 0xd9, 0xda,
    0xe2, 0xe3, 0xe4, 0xe5, 0xe6, 0xe7, 0xe8, 0xe9, 0xea, 0xf2, 0xf3, 0xf4, 0xf5, 0xf6, 0xf7, 0xf8, 0xf9, 0xfa};

/* --------------------------------------------------------------- helpers */

void oracle_jpeg_quant_table(int quality, int chroma, int* q /*[64] natural*/) {
    if (quality < 1) quality = 1;
    if (quality > 100) quality = 100;
    const int scale = quality < 50 ? 5000 / quality : 200 - 2 * quality;
    const int* base = chroma ? kBaseChroma : kBaseLuma;
    for (int i = 0; i < 64; ++i) {
        int v = (base[i] * scale + 50) / 100;
        q[i] = v < 1 ? 1 : (v > 255 ? 255 : v);
    }
}

/* Canonical codes from code-length counts (Annex C): code[symbol], size[symbol]. */
static void build_codes(const uint8_t* bits, const uint8_t* vals, int nvals, uint16_t* code, uint8_t* size) {
    int k = 0;
    uint32_t c = 0;
    memset(size, 0, 256);
    for (int len = 1; len <= 16; ++len) {
        for (int i = 0; i < bits[len - 1]; ++i) {
            code[vals[k]] = (uint16_t)c;
            size[vals[k]] = (uint8_t)len;
            ++k;
            ++c;
        }
        c <<= 1;
    }
    (void)nvals;
}

/* The T.81 FDCT weights in 13-bit fixed point: w[u][x] = round(2^13 C(u)/2 cos((2x+1)u pi/16)). */
static void dct_weights(int w[8][8]) {
    for (int u = 0; u < 8; ++u)
        for (int x = 0; x < 8; ++x) {
            const double cu = u == 0 ? 1.0 / sqrt(2.0) : 1.0;
            const double v = 8192.0 * 0.5 * cu * cos((2.0 * x + 1.0) * u * M_PI / 16.0);
            w[u][x] = (int)floor(v + 0.5);
        }
}

/* 8x8 block of level-shifted samples s[y][x] -> coefficients scaled by 2^16 (natural order). */
static void fdct_fixed(const int w[8][8], const int s[64], int32_t c[64]) {
    int32_t r[64];
    for (int y = 0; y < 8; ++y)
        for (int u = 0; u < 8; ++u) {
            int32_t acc = 0;
            for (int x = 0; x < 8; ++x) acc += w[u][x] * s[y * 8 + x];
            r[y * 8 + u] = (acc + 512) >> 10;   /* floor((acc + 2^9) / 2^10) */
        }
    for (int v = 0; v < 8; ++v)
        for (int u = 0; u < 8; ++u) {
            int32_t acc = 0;
            for (int y = 0; y < 8; ++y) acc += w[v][y] * r[y * 8 + u];
            c[v * 8 + u] = acc;
        }
}

/* Coefficient scaled by 2^16 divided by the quantizer step, nearest, halves away from zero. */
static int quantize(int32_t c, int q) {
    const int64_t den = (int64_t)q << 16;
    const int64_t a = c < 0 ? -(int64_t)c : (int64_t)c;
    const int64_t m = (a + (den >> 1)) / den;
    return (int)(c < 0 ? -m : m);
}

void oracle_jpeg_fdct_fixed(const int* s /*[64]*/, int* out /*[64], scaled by 2^16*/) {
    int w[8][8];
    dct_weights(w);
    int32_t c[64];
    fdct_fixed(w, s, c);
    for (int i = 0; i < 64; ++i) out[i] = c[i];
}

/* The FDCT definition in double precision (Annex A.3.3), for the pins. */
void oracle_jpeg_fdct_exact(const int* s, double* out) {
    for (int v = 0; v < 8; ++v)
        for (int u = 0; u < 8; ++u) {
            const double cu = u == 0 ? 1.0 / sqrt(2.0) : 1.0, cv = v == 0 ? 1.0 / sqrt(2.0) : 1.0;
            double acc = 0.0;
            for (int y = 0; y < 8; ++y)
                for (int x = 0; x < 8; ++x)
                    acc += s[y * 8 + x] * cos((2.0 * x + 1.0) * u * M_PI / 16.0) * cos((2.0 * y + 1.0) * v * M_PI / 16.0);
            out[v * 8 + u] = 0.25 * cu * cv * acc;
        }
}

/* JFIF colour conversion of one pixel (weights x 65536, rounded). */
static void rgb_to_ycc(int r, int g, int b, int* y, int* cb, int* cr) {
    int Y = (19595 * r + 38470 * g + 7471 * b + 32768) >> 16;
    int Cb = (-11058 * r - 21710 * g + 32768 * b + (128 << 16) + 32768) >> 16;
    int Cr = (32768 * r - 27439 * g - 5329 * b + (128 << 16) + 32768) >> 16;
    *y = Y > 255 ? 255 : Y;
    *cb = Cb > 255 ? 255 : Cb;
    *cr = Cr > 255 ? 255 : Cr;
}

/* ---------------------------------------------------------------- writer */

typedef struct {
    uint8_t* buf;
    size_t cap, len;
    uint64_t acc;   /* bit accumulator, msb first */
    int nbits;
    int overflow;
} Writer;

static void put_byte(Writer* w, uint8_t b) {
    if (w->len < w->cap) w->buf[w->len] = b; else w->overflow = 1;
    w->len++;
}
static void put_bits(Writer* w, uint32_t v, int n) {   /* entropy-coded bits, stuffed */
    if (n == 0) return;
    w->acc = (w->acc << n) | (v & ((1u << n) - 1u));
    w->nbits += n;
    while (w->nbits >= 8) {
        const uint8_t b = (uint8_t)(w->acc >> (w->nbits - 8));
        put_byte(w, b);
        if (b == 0xFF) put_byte(w, 0x00);
        w->nbits -= 8;
    }
}
static void flush_bits(Writer* w) {   /* pad the last byte with 1s */
    if (w->nbits > 0) put_bits(w, 0x7F, 8 - w->nbits);
    w->acc = 0;
    w->nbits = 0;
}
static void put_u16(Writer* w, int v) {
    put_byte(w, (uint8_t)(v >> 8));
    put_byte(w, (uint8_t)v);
}

static int category(int v) {
    int a = v < 0 ? -v : v, n = 0;
    while (a) { ++n; a >>= 1; }
    return n;
}

static void encode_block(Writer* w, const int* zz, int* pred, const uint16_t* dcc, const uint8_t* dcs,
                         const uint16_t* acc, const uint8_t* acs) {
    const int diff = zz[0] - *pred;
    *pred = zz[0];
    int n = category(diff);
    put_bits(w, dcc[n], dcs[n]);
    if (n) put_bits(w, (uint32_t)(diff < 0 ? diff - 1 : diff), n);
    int run = 0;
    for (int k = 1; k < 64; ++k) {
        const int v = zz[k];
        if (v == 0) { ++run; continue; }
        while (run > 15) { put_bits(w, acc[0xF0], acs[0xF0]); run -= 16; }
        n = category(v);
        const int sym = (run << 4) | n;
        put_bits(w, acc[sym], acs[sym]);
        put_bits(w, (uint32_t)(v < 0 ? v - 1 : v), n);
        run = 0;
    }
    if (run > 0) put_bits(w, acc[0x00], acs[0x00]);
}

static void put_dht(Writer* w, int cls, int id, const uint8_t* bits, const uint8_t* vals, int nvals) {
    put_u16(w, 0xFFC4);
    put_u16(w, 2 + 1 + 16 + nvals);
    put_byte(w, (uint8_t)((cls << 4) | id));
    for (int i = 0; i < 16; ++i) put_byte(w, bits[i]);
    for (int i = 0; i < nvals; ++i) put_byte(w, vals[i]);
}

/* Encode an RGBA8 image; returns the file length (which may exceed cap: then
 * nothing beyond cap was written).  restart: MCUs per restart interval (0: none). */
int64_t oracle_jpeg_encode(const uint8_t* rgba, int width, int height, int quality, int restart, uint8_t* out,
                           int64_t cap) {
    if (width < 1 || height < 1 || width > 65535 || height > 65535) return -1;
    Writer w = {out, (size_t)(cap < 0 ? 0 : cap), 0, 0, 0, 0};
    int ql[64], qc[64];
    oracle_jpeg_quant_table(quality, 0, ql);
    oracle_jpeg_quant_table(quality, 1, qc);
    int wts[8][8];
    dct_weights(wts);
    uint16_t dc0c[256], dc1c[256], ac0c[256], ac1c[256];
    uint8_t dc0s[256], dc1s[256], ac0s[256], ac1s[256];
    build_codes(kDcLumaBits, kDcVals, 12, dc0c, dc0s);
    build_codes(kDcChromaBits, kDcVals, 12, dc1c, dc1s);
    build_codes(kAcLumaBits, kAcLumaVals, 162, ac0c, ac0s);
    build_codes(kAcChromaBits, kAcChromaVals, 162, ac1c, ac1s);

    /* headers: SOI, APP0 (JFIF 1.01), DQT, SOF0, DHT x4, DRI, SOS */
    put_u16(&w, 0xFFD8);
    put_u16(&w, 0xFFE0);
    put_u16(&w, 16);
    const uint8_t jfif[14] = {'J', 'F', 'I', 'F', 0, 1, 1, 0, 0, 1, 0, 1, 0, 0};
    for (int i = 0; i < 14; ++i) put_byte(&w, jfif[i]);
    for (int t = 0; t < 2; ++t) {
        put_u16(&w, 0xFFDB);
        put_u16(&w, 67);
        put_byte(&w, (uint8_t)t);
        const int* q = t ? qc : ql;
        for (int k = 0; k < 64; ++k) put_byte(&w, (uint8_t)q[kZigzag[k]]);
    }
    put_u16(&w, 0xFFC0);
    put_u16(&w, 17);
    put_byte(&w, 8);
    put_u16(&w, height);
    put_u16(&w, width);
    put_byte(&w, 3);
    const uint8_t comps[9] = {1, 0x22, 0, 2, 0x11, 1, 3, 0x11, 1};
    for (int i = 0; i < 9; ++i) put_byte(&w, comps[i]);
    put_dht(&w, 0, 0, kDcLumaBits, kDcVals, 12);
    put_dht(&w, 1, 0, kAcLumaBits, kAcLumaVals, 162);
    put_dht(&w, 0, 1, kDcChromaBits, kDcVals, 12);
    put_dht(&w, 1, 1, kAcChromaBits, kAcChromaVals, 162);
    if (restart > 0) {
        put_u16(&w, 0xFFDD);
        put_u16(&w, 4);
        put_u16(&w, restart);
    }
    put_u16(&w, 0xFFDA);
    put_u16(&w, 12);
    put_byte(&w, 3);
    const uint8_t sos[6] = {1, 0x00, 2, 0x11, 3, 0x11};
    for (int i = 0; i < 6; ++i) put_byte(&w, sos[i]);
    put_byte(&w, 0);
    put_byte(&w, 63);
    put_byte(&w, 0);

    /* MCUs in raster order */
    const int mw = (width + 15) / 16, mh = (height + 15) / 16;
    int pred[3] = {0, 0, 0};
    int done_in_interval = 0, rst = 0;
    for (int my = 0; my < mh; ++my)
        for (int mx = 0; mx < mw; ++mx) {
            if (restart > 0 && done_in_interval == restart) {
                flush_bits(&w);
                put_byte(&w, 0xFF);
                put_byte(&w, (uint8_t)(0xD0 + (rst & 7)));
                ++rst;
                pred[0] = pred[1] = pred[2] = 0;
                done_in_interval = 0;
            }
            int Y[256], Cb[256], Cr[256];
            for (int j = 0; j < 16; ++j)
                for (int i = 0; i < 16; ++i) {
                    int x = mx * 16 + i, y = my * 16 + j;
                    if (x >= width) x = width - 1;
                    if (y >= height) y = height - 1;
                    const uint8_t* p = rgba + 4 * ((size_t)y * width + x);
                    rgb_to_ycc(p[0], p[1], p[2], &Y[j * 16 + i], &Cb[j * 16 + i], &Cr[j * 16 + i]);
                }
            int s[64], zz[64];
            int32_t c[64];
            for (int b = 0; b < 4; ++b) {
                const int ox = (b & 1) * 8, oy = (b >> 1) * 8;
                for (int j = 0; j < 8; ++j)
                    for (int i = 0; i < 8; ++i) s[j * 8 + i] = Y[(oy + j) * 16 + ox + i] - 128;
                fdct_fixed(wts, s, c);
                for (int k = 0; k < 64; ++k) zz[k] = quantize(c[kZigzag[k]], ql[kZigzag[k]]);
                encode_block(&w, zz, &pred[0], dc0c, dc0s, ac0c, ac0s);
            }
            for (int comp = 0; comp < 2; ++comp) {
                const int* src = comp ? Cr : Cb;
                for (int j = 0; j < 8; ++j)
                    for (int i = 0; i < 8; ++i) {
                        const int sum = src[(2 * j) * 16 + 2 * i] + src[(2 * j) * 16 + 2 * i + 1] +
                                        src[(2 * j + 1) * 16 + 2 * i] + src[(2 * j + 1) * 16 + 2 * i + 1];
                        s[j * 8 + i] = ((sum + 2) >> 2) - 128;
                    }
                fdct_fixed(wts, s, c);
                for (int k = 0; k < 64; ++k) zz[k] = quantize(c[kZigzag[k]], qc[kZigzag[k]]);
                encode_block(&w, zz, &pred[1 + comp], dc1c, dc1s, ac1c, ac1s);
            }
            ++done_in_interval;
        }
    flush_bits(&w);
    put_u16(&w, 0xFFD9);
    return (int64_t)w.len;
}
