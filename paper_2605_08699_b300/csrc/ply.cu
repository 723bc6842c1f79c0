// 3DGS PLY models (Sec. 4.1 and Sec. 5.1, "PLY Model and Primitives"): each
// scene file holds one vertex per Gaussian with its centre, log-scales,
// rotation quaternion, opacity logit and SH coefficients.  The header is
// parsed on the host; the vertex block is streamed through two pinned buffers
// into device memory and de-interleaved there (k_ply_gather) into the raw
// attribute arrays that scene packing activates.  Big-endian bodies are
// byte-swapped and ASCII bodies tokenised on the host first, into a record
// layout the same kernel reads.
#include <sys/stat.h>

#include <algorithm>
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "pipeline.cuh"

namespace tigas {

namespace {

constexpr size_t kMaxHeader = 1 << 20;       // bytes of header text accepted
constexpr size_t kStreamChunk = 32u << 20;   // pinned staging buffer size

struct PlyGatherMap {
    uint32_t offset[kPlyFields];
    uint8_t type[kPlyFields];
};

__device__ __forceinline__ uint32_t le_u32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

__device__ __forceinline__ float ply_value(const uint8_t* p, int t) {
    switch (t) {
        case kPlyI8: return (float)(int8_t)p[0];
        case kPlyU8: return (float)p[0];
        case kPlyI16: return (float)(int16_t)(uint16_t)(p[0] | (p[1] << 8));
        case kPlyU16: return (float)(uint16_t)(p[0] | (p[1] << 8));
        case kPlyI32: return (float)(int32_t)le_u32(p);
        case kPlyU32: return (float)le_u32(p);
        case kPlyF32: return __uint_as_float(le_u32(p));
        case kPlyF64: {
            unsigned long long u = (unsigned long long)le_u32(p) | ((unsigned long long)le_u32(p + 4) << 32);
            return __double2float_rn(__longlong_as_double((long long)u));
        }
        default: return 0.0f;
    }
}

// One thread per (vertex, field): consecutive threads read consecutive fields
// of a record, so a warp's loads stay within one or two records.
__global__ void __launch_bounds__(256)
k_ply_gather(const uint8_t* __restrict__ rows, uint64_t n, uint32_t row_bytes, PlyGatherMap map,
             float* __restrict__ means, float* __restrict__ log_scales, float* __restrict__ quats,
             float* __restrict__ logits, float* __restrict__ sh) {
    const uint64_t total = n * kPlyFields;
    for (uint64_t o = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = o / kPlyFields;
        const int f = (int)(o - i * kPlyFields);
        const int t = map.type[f];
        const float v = t == kPlyAbsent ? 0.0f : ply_value(rows + i * row_bytes + map.offset[f], t);
        if (f < 3) means[3 * i + f] = v;
        else if (f < 6) log_scales[3 * i + (f - 3)] = v;
        else if (f < 10) quats[4 * i + (f - 6)] = v;
        else if (f == 10) logits[i] = v;
        else sh[48 * i + (f - 11)] = v;
    }
}

int type_code(const std::string& s, int* bytes) {
    struct T { const char* a; const char* b; int code; int size; };
    static const T table[] = {{"char", "int8", kPlyI8, 1},     {"uchar", "uint8", kPlyU8, 1},
                              {"short", "int16", kPlyI16, 2},  {"ushort", "uint16", kPlyU16, 2},
                              {"int", "int32", kPlyI32, 4},    {"uint", "uint32", kPlyU32, 4},
                              {"float", "float32", kPlyF32, 4}, {"double", "float64", kPlyF64, 8}};
    for (const T& t : table)
        if (s == t.a || s == t.b) {
            *bytes = t.size;
            return t.code;
        }
    return -1;
}

std::vector<std::string> split(const std::string& line) {
    std::vector<std::string> out;
    size_t i = 0;
    while (i < line.size()) {
        while (i < line.size() && (line[i] == ' ' || line[i] == '\t' || line[i] == '\r')) ++i;
        size_t j = i;
        while (j < line.size() && line[j] != ' ' && line[j] != '\t' && line[j] != '\r') ++j;
        if (j > i) out.push_back(line.substr(i, j - i));
        i = j;
    }
    return out;
}

struct File {
    FILE* f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

Status io_error(const char* path, const char* what) {
    return {TIGAS_ERR_IO, std::string(what) + " " + path + ": " + strerror(errno)};
}

Status bad(const char* path, const std::string& what) { return {TIGAS_ERR_INVALID, std::string(path) + ": " + what}; }

// Field index of a 3DGS property name (the f_rest_* ones are placed once the
// SH degree is known); -1 when the property is not one the scene uses.
int fixed_field(const std::string& name) {
    static const char* names[11] = {"x", "y", "z", "scale_0", "scale_1", "scale_2",
                                    "rot_0", "rot_1", "rot_2", "rot_3", "opacity"};
    for (int k = 0; k < 11; ++k)
        if (name == names[k]) return k;
    for (int c = 0; c < 3; ++c)
        if (name == "f_dc_" + std::to_string(c)) return 11 + c;
    return -1;
}

struct Element {
    std::string name;
    uint64_t count = 0;
    uint32_t bytes = 0;      // binary record size
    bool has_list = false;
    std::vector<std::string> props;
    std::vector<uint8_t> types;
    std::vector<uint32_t> offsets;
};

}  // namespace

Status ply_probe(const char* path, PlyLayout* out) {
    File file;
    file.f = fopen(path, "rb");
    if (!file.f) return io_error(path, "cannot open");
    struct stat sb;
    if (fstat(fileno(file.f), &sb) != 0) return io_error(path, "cannot stat");
    PlyLayout lay;
    lay.file_bytes = (uint64_t)sb.st_size;

    // Header lines up to "end_header".
    std::vector<std::string> lines;
    std::string cur;
    size_t consumed = 0;
    bool ended = false;
    int ch;
    while (consumed < kMaxHeader && (ch = fgetc(file.f)) != EOF) {
        ++consumed;
        if (ch == '\n') {
            if (!cur.empty() && cur.back() == '\r') cur.pop_back();
            lines.push_back(cur);
            if (cur == "end_header") {
                ended = true;
                break;
            }
            cur.clear();
        } else {
            cur.push_back((char)ch);
        }
    }
    if (lines.empty() || lines[0] != "ply") return bad(path, "not a PLY file (no 'ply' magic line)");
    if (!ended) return bad(path, "header has no end_header line");

    bool have_format = false;
    std::vector<Element> elems;
    for (size_t li = 1; li + 1 < lines.size(); ++li) {
        std::vector<std::string> tok = split(lines[li]);
        if (tok.empty() || tok[0] == "comment" || tok[0] == "obj_info") continue;
        if (tok[0] == "format") {
            if (tok.size() < 2) return bad(path, "malformed format line");
            if (tok[1] == "binary_little_endian") lay.format = kPlyBinaryLE;
            else if (tok[1] == "binary_big_endian") lay.format = kPlyBinaryBE;
            else if (tok[1] == "ascii") lay.format = kPlyAscii;
            else return bad(path, "unknown format '" + tok[1] + "'");
            have_format = true;
        } else if (tok[0] == "element") {
            if (tok.size() != 3) return bad(path, "malformed element line");
            char* end = nullptr;
            errno = 0;
            unsigned long long c = strtoull(tok[2].c_str(), &end, 10);
            if (errno || !end || *end || tok[2][0] == '-') return bad(path, "bad element count '" + tok[2] + "'");
            Element e;
            e.name = tok[1];
            e.count = c;
            elems.push_back(e);
        } else if (tok[0] == "property") {
            if (elems.empty()) return bad(path, "property before any element");
            Element& e = elems.back();
            if (tok.size() == 5 && tok[1] == "list") {
                e.has_list = true;
                e.props.push_back(tok[4]);
                e.types.push_back(kPlyAbsent);
                e.offsets.push_back(0);
                continue;
            }
            if (tok.size() != 3) return bad(path, "malformed property line");
            int size = 0;
            int code = type_code(tok[1], &size);
            if (code < 0) return bad(path, "unknown property type '" + tok[1] + "'");
            e.props.push_back(tok[2]);
            e.types.push_back((uint8_t)code);
            e.offsets.push_back(e.bytes);
            e.bytes += (uint32_t)size;
        } else {
            return bad(path, "unknown header keyword '" + tok[0] + "'");
        }
    }
    if (!have_format) return bad(path, "header has no format line");

    // Locate the vertex element and what precedes it.
    uint64_t pre_bytes = 0, pre_lines = 0;
    const Element* vert = nullptr;
    for (const Element& e : elems) {
        if (e.name == "vertex") {
            vert = &e;
            break;
        }
        if (lay.format != kPlyAscii && e.has_list)
            return bad(path, "list property in element '" + e.name + "' before the vertex element");
        pre_bytes += e.count * e.bytes;
        pre_lines += e.count;
    }
    if (!vert) return bad(path, "no vertex element");
    if (vert->has_list) return bad(path, "list property in the vertex element");
    if (vert->count < 1 || vert->count > (1ull << 27)) return bad(path, "vertex count out of 1..2^27");
    lay.n = vert->count;
    lay.row_bytes = vert->bytes;
    lay.prop_type = vert->types;
    lay.prop_offset = vert->offsets;
    lay.body_offset = consumed + (lay.format == kPlyAscii ? 0 : pre_bytes);
    lay.skip_lines = lay.format == kPlyAscii ? pre_lines : 0;

    // Fields: fixed names, then f_rest_0 .. f_rest_{3M-1}.
    for (int f = 0; f < kPlyFields; ++f) lay.field_prop[f] = -1;
    std::vector<int> rest;   // property index of f_rest_k
    for (size_t p = 0; p < vert->props.size(); ++p) {
        const std::string& name = vert->props[p];
        int f = fixed_field(name);
        if (f >= 0) {
            if (lay.field_prop[f] >= 0) return bad(path, "duplicate property '" + name + "'");
            lay.field_prop[f] = (int32_t)p;
        } else if (name.compare(0, 7, "f_rest_") == 0) {
            char* end = nullptr;
            long k = strtol(name.c_str() + 7, &end, 10);
            if (!end || *end || k < 0 || k >= 45) return bad(path, "bad SH property '" + name + "'");
            if ((int)rest.size() <= k) rest.resize(k + 1, -1);
            if (rest[k] >= 0) return bad(path, "duplicate property '" + name + "'");
            rest[k] = (int)p;
        }
    }
    static const char* required[14] = {"x", "y", "z", "scale_0", "scale_1", "scale_2", "rot_0",
                                       "rot_1", "rot_2", "rot_3", "opacity", "f_dc_0", "f_dc_1", "f_dc_2"};
    for (int f = 0; f < 14; ++f)
        if (lay.field_prop[f] < 0) return bad(path, std::string("missing vertex property '") + required[f] + "'");
    const int n_rest = (int)rest.size();
    int degree = -1;
    for (int d = 0; d <= 3; ++d)
        if (n_rest == 3 * ((d + 1) * (d + 1) - 1)) degree = d;
    if (degree < 0) return bad(path, "f_rest_* count " + std::to_string(n_rest) + " is not 0, 9, 24 or 45");
    for (int k = 0; k < n_rest; ++k)
        if (rest[k] < 0) return bad(path, "f_rest_" + std::to_string(k) + " is missing");
    lay.sh_degree = degree;
    const int M = (degree + 1) * (degree + 1) - 1;
    for (int c = 0; c < 3; ++c)
        for (int j = 0; j < M; ++j) lay.field_prop[11 + 3 * (j + 1) + c] = rest[c * M + j];

    if (lay.format != kPlyAscii && lay.body_offset + lay.n * lay.row_bytes > lay.file_bytes)
        return bad(path, "file is shorter than its vertex block (truncated)");
    *out = std::move(lay);
    return {};
}

namespace {

// Host record buffer of an ASCII body: every vertex property as float64.
Status ascii_records(const char* path, FILE* f, const PlyLayout& lay, std::vector<double>* rec) {
    const size_t np = lay.prop_type.size();
    if (fseeko(f, (off_t)lay.body_offset, SEEK_SET) != 0) return io_error(path, "cannot seek");
    std::string text;
    text.resize(lay.file_bytes - lay.body_offset);
    if (!text.empty() && fread(&text[0], 1, text.size(), f) != text.size()) return io_error(path, "cannot read");
    const char* p = text.c_str();
    const char* end = p + text.size();
    for (uint64_t s = 0; s < lay.skip_lines; ++s) {
        const char* nl = (const char*)memchr(p, '\n', end - p);
        if (!nl) return bad(path, "ascii body ends before the vertex element");
        p = nl + 1;
    }
    rec->resize(lay.n * np);
    for (uint64_t i = 0; i < lay.n; ++i) {
        for (size_t k = 0; k < np; ++k) {
            char* q = nullptr;
            double v = strtod(p, &q);
            if (q == p) return bad(path, "ascii vertex " + std::to_string(i) + " has too few values");
            (*rec)[i * np + k] = v;
            p = q;
        }
        while (p < end && *p != '\n') {
            if (*p != ' ' && *p != '\t' && *p != '\r')
                return bad(path, "ascii vertex " + std::to_string(i) + " has extra values");
            ++p;
        }
        if (p < end) ++p;
    }
    return {};
}

void swap_record_bytes(uint8_t* rows, uint64_t n, const PlyLayout& lay) {
    for (uint64_t i = 0; i < n; ++i) {
        uint8_t* r = rows + i * lay.row_bytes;
        for (size_t p = 0; p < lay.prop_type.size(); ++p) {
            const int t = lay.prop_type[p];
            const int size = t <= kPlyU8 ? 1 : t <= kPlyU16 ? 2 : t == kPlyF64 ? 8 : 4;
            std::reverse(r + lay.prop_offset[p], r + lay.prop_offset[p] + size);
        }
    }
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};
struct PinnedBuf {
    void* p = nullptr;
    ~PinnedBuf() {
        if (p) cudaFreeHost(p);
    }
};
struct Events {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Events() {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
};

// Binary little-endian body: file -> pinned chunk -> device, double-buffered
// so that reading chunk k+1 overlaps the copy of chunk k.
Status stream_le(const char* path, FILE* f, uint64_t bytes, uint8_t* dst, cudaStream_t st) {
    PinnedBuf pin[2];
    Events ev;
    const size_t chunk = (size_t)std::min<uint64_t>(kStreamChunk, bytes);
    for (int b = 0; b < 2; ++b) {
        TIGAS_CUDA_TRY(pinned_alloc(&pin[b].p, chunk));
        TIGAS_CUDA_TRY(cudaEventCreateWithFlags(&ev.e[b], cudaEventDisableTiming));
    }
    uint64_t done = 0;
    for (int k = 0; done < bytes; ++k) {
        const int b = k & 1;
        const size_t len = (size_t)std::min<uint64_t>(chunk, bytes - done);
        if (k >= 2) TIGAS_CUDA_TRY(cudaEventSynchronize(ev.e[b]));
        if (fread(pin[b].p, 1, len, f) != len) return io_error(path, "cannot read vertex block");
        TIGAS_CUDA_TRY(cudaMemcpyAsync(dst + done, pin[b].p, len, cudaMemcpyHostToDevice, st));
        TIGAS_CUDA_TRY(cudaEventRecord(ev.e[b], st));
        done += len;
    }
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    return {};
}

}  // namespace

Status ply_decode(const char* path, const PlyLayout& lay, float* means, float* log_scales, float* quats,
                  float* logits, float* sh, cudaStream_t st) {
    File file;
    file.f = fopen(path, "rb");
    if (!file.f) return io_error(path, "cannot open");
    PlyGatherMap map;
    uint32_t row_bytes = lay.row_bytes;
    DevBuf rows;
    if (lay.format == kPlyAscii) {
        std::vector<double> rec;
        Status s = ascii_records(path, file.f, lay, &rec);
        if (!s.ok()) return s;
        row_bytes = (uint32_t)(8 * lay.prop_type.size());
        TIGAS_CUDA_TRY(device_alloc(&rows.p, rec.size() * 8));
        TIGAS_CUDA_TRY(cudaMemcpy(rows.p, rec.data(), rec.size() * 8, cudaMemcpyHostToDevice));
        for (int f = 0; f < kPlyFields; ++f) {
            const int p = lay.field_prop[f];
            map.offset[f] = p < 0 ? 0u : (uint32_t)(8 * p);
            map.type[f] = p < 0 ? (uint8_t)kPlyAbsent : (uint8_t)kPlyF64;
        }
    } else {
        const uint64_t bytes = lay.n * lay.row_bytes;
        TIGAS_CUDA_TRY(device_alloc(&rows.p, bytes));
        if (fseeko(file.f, (off_t)lay.body_offset, SEEK_SET) != 0) return io_error(path, "cannot seek");
        if (lay.format == kPlyBinaryLE) {
            Status s = stream_le(path, file.f, bytes, (uint8_t*)rows.p, st);
            if (!s.ok()) return s;
        } else {
            std::vector<uint8_t> host(bytes);
            if (fread(host.data(), 1, bytes, file.f) != bytes) return io_error(path, "cannot read vertex block");
            swap_record_bytes(host.data(), lay.n, lay);
            TIGAS_CUDA_TRY(cudaMemcpy(rows.p, host.data(), bytes, cudaMemcpyHostToDevice));
        }
        for (int f = 0; f < kPlyFields; ++f) {
            const int p = lay.field_prop[f];
            map.offset[f] = p < 0 ? 0u : lay.prop_offset[p];
            map.type[f] = p < 0 ? (uint8_t)kPlyAbsent : lay.prop_type[p];
        }
    }
    const uint64_t total = lay.n * kPlyFields;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)kSmCount * 16);
    k_ply_gather<<<grid, 256, 0, st>>>((const uint8_t*)rows.p, lay.n, row_bytes, map, means, log_scales, quats,
                                       logits, sh);
    TIGAS_LAUNCHED();
    TIGAS_CUDA_TRY(cudaGetLastError());
    TIGAS_CUDA_TRY(cudaStreamSynchronize(st));
    return {};
}

Status scene_load_ply(const char* path, int storage, const float bg[3], Scene** out) {
    *out = nullptr;
    PlyLayout lay;
    Status s = ply_probe(path, &lay);
    if (!s.ok()) return s;
    const uint64_t n = lay.n;
    DevBuf raw;
    TIGAS_CUDA_TRY(device_alloc(&raw.p, n * kPlyFields * sizeof(float)));
    float* p = (float*)raw.p;
    float *m = p, *ls = m + 3 * n, *q = ls + 3 * n, *op = q + 4 * n, *sh = op + n;
    cudaStream_t st = nullptr;
    TIGAS_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    s = ply_decode(path, lay, m, ls, q, op, sh, st);
    if (s.ok()) s = scene_create(m, ls, q, op, sh, (uint32_t)n, lay.sh_degree, storage, bg, st, out);
    cudaStreamDestroy(st);
    return s;
}

}  // namespace tigas
