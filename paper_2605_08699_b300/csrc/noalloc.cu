// tigas_sort_pairs_u64_noalloc: the device radix sort with its scratch in a
// fixed, file-scope device array instead of library-allocated workspace.
//
// Some callers cannot let this library call cudaMalloc: applications that own
// every byte of device memory through their own pools or budgets, and hosts
// whose threads must not take the implicit device-wide synchronisation that
// cudaMalloc/cudaFree can cause.  This entry point serves them: the caller
// passes inputs and outputs, and the sort's ping-pong buffers, digit tables
// and scan scratch live in g_sort_scratch below, which every GPU that loads
// the library holds until the process exits.
//
// The sort returns once its work is queued, so a look-back wait that ran out
// (the sort's bounded spin, see sort.cu) cannot be reported by the call
// itself.  Every call ORs that event into one sticky word at the end of the
// scratch (zero when the library is loaded); tigas_sort_noalloc_check waits
// for the caller's stream and reads and clears it.
#include <mutex>

#include "kernels.cuh"

#define TIGAS_API extern "C" __attribute__((visibility("default")))

namespace tigas {
tigas_status fail(const Status& s);
tigas_status fail(tigas_status code, const std::string& msg);
}  // namespace tigas

namespace {

// Largest n accepted: 2^20 pairs.  Scratch: alternate keys (8 B) and values
// (4 B) per pair, plus the sort's digit tables and scan scratch, plus the
// sticky timeout word (in its own 256-byte block).
constexpr uint64_t kMaxPairs = 1ull << 20;
constexpr size_t kAltKeyBytes = kMaxPairs * 8;
constexpr size_t kAltValBytes = kMaxPairs * 4;
constexpr size_t kTableBytes = 1u << 22;   // >= radix_tmp_words(kMaxPairs) * 4 (checked at set-up)
constexpr size_t kFlagOffset = kAltKeyBytes + kAltValBytes + kTableBytes;
constexpr size_t kScratchBytes = kFlagOffset + 256;

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[tigas::kMaxDevices] = {};

// Device address of g_sort_scratch on the current device, looked up once per
// device.  (In host code the array's name is only a host-side stand-in.)
// A non-null stream must belong to the current device: the scratch address
// is that device's.
tigas::Status scratch_for_current_device(cudaStream_t stream, unsigned char** out) {
    int dev = 0;
    TIGAS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= tigas::kMaxDevices) return {TIGAS_ERR_INVALID, "device ordinal out of range"};
    if (stream) {
        int sdev = -1;
        TIGAS_CUDA_TRY(cudaStreamGetDevice(stream, &sdev));
        if (sdev != dev)
            return {TIGAS_ERR_INVALID, "cuda_stream belongs to device " + std::to_string(sdev) +
                                           ", the current device is " + std::to_string(dev)};
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        if (tigas::radix_tmp_words(kMaxPairs) * 4 > kTableBytes)
            return {TIGAS_ERR_CUDA, "static sort scratch too small for its maximum"};
        if (tigas::debug_lookback_words() * 4 > kFlagOffset)
            return {TIGAS_ERR_CUDA, "static sort scratch too small for the look-back probe"};
        void* p = nullptr;
        TIGAS_CUDA_TRY(cudaGetSymbolAddress(&p, g_sort_scratch));
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return {};
}

uint32_t* timeout_word(unsigned char* scratch) { return reinterpret_cast<uint32_t*>(scratch + kFlagOffset); }

}  // namespace

using namespace tigas;

TIGAS_API tigas_status tigas_sort_pairs_u64_noalloc(const uint64_t* keys_in, const uint32_t* values_in,
                                                    uint64_t* keys_out, uint32_t* values_out, uint64_t n,
                                                    int begin_bit, int end_bit, void* cuda_stream) {
    set_error("");
    if (n > kMaxPairs)
        return fail(TIGAS_ERR_INVALID, "n = " + std::to_string(n) + " exceeds the static scratch maximum of " +
                                           std::to_string(kMaxPairs) + " pairs");
    if (n > 0 && (!keys_in || !values_in || !keys_out || !values_out)) return fail(TIGAS_ERR_INVALID, "null buffer");
    if (begin_bit < 0 || end_bit > 64 || begin_bit >= end_bit) return fail(TIGAS_ERR_INVALID, "bad bit range");
    if (n == 0) return TIGAS_OK;
    if (keys_in == keys_out || values_in == values_out) return fail(TIGAS_ERR_INVALID, "in and out must differ");
    unsigned char* scratch = nullptr;
    Status s = scratch_for_current_device((cudaStream_t)cuda_stream, &scratch);
    if (!s.ok()) return fail(s);
    // Nothing here must start at zero: every scratch word the sort reads is
    // written earlier by the same call (digit tables by the histogram kernel,
    // ping-pong buffers by the previous pass).  The timeout word is only ORed.
    auto* alt_k = reinterpret_cast<uint64_t*>(scratch);
    auto* alt_v = reinterpret_cast<uint32_t*>(scratch + kAltKeyBytes);
    auto* tmp = reinterpret_cast<uint32_t*>(scratch + kAltKeyBytes + kAltValBytes);
    s = radix_sort<uint64_t>(keys_in, values_in, alt_k, alt_v, keys_out, values_out, n, nullptr, begin_bit, end_bit,
                             tmp, (cudaStream_t)cuda_stream, nullptr, timeout_word(scratch));
    if (!s.ok()) return fail(s);
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_sort_noalloc_check(void* cuda_stream) {
    set_error("");
    unsigned char* scratch = nullptr;
    Status s = scratch_for_current_device((cudaStream_t)cuda_stream, &scratch);
    if (!s.ok()) return fail(s);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    uint32_t word = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&word, timeout_word(scratch), sizeof(word), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && word != 0) e = cudaMemset(timeout_word(scratch), 0, sizeof(word));
    if (e != cudaSuccess) return fail(TIGAS_ERR_CUDA, std::string("noalloc sort check: ") + cudaGetErrorString(e));
    if (word & kSortTimeoutFlag)
        return fail(TIGAS_ERR_TIMEOUT, "a radix sort look-back wait of an allocation-free sort ran out");
    return TIGAS_OK;
}

TIGAS_API tigas_status tigas_debug_sort_noalloc_wait_timeout(int spin_limit, void* cuda_stream) {
    set_error("");
    unsigned char* scratch = nullptr;
    Status s = scratch_for_current_device((cudaStream_t)cuda_stream, &scratch);
    if (!s.ok()) return fail(s);
    // the probe runs in the scratch's ping-pong region and ORs into the sticky word
    s = debug_lookback_enqueue(spin_limit, reinterpret_cast<uint32_t*>(scratch), timeout_word(scratch),
                               (cudaStream_t)cuda_stream);
    if (!s.ok()) return fail(s);
    return TIGAS_OK;
}
