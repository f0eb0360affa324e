// vqnqs_compress_rows_noalloc: the (I, V) compression of vqnqs_compress_rows
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need this step: code running while a stream is being captured
// into a CUDA graph, code embedded in a host application whose device memory
// is owned by someone else, or a hook that must not grow the footprint.  This
// entry point takes only the caller's inputs and outputs; its hash table lives
// in the file-scope array below, which every GPU that loads the library holds
// until the process exits.
//
// Limits and sharing:
//  - at most VQNQS_NOALLOC_MAX_ROWS = 2^18 rows per call (the table has 2^19
//    slots, so a load of at most 1/2 keeps every probe short);
//  - every call on a device uses the same array; each call clears the part it
//    uses first, so the previous call's contents never leak into a result, but
//    calls whose kernels overlap on the GPU (different streams, or different
//    host threads on one device) race on the table and give wrong results;
//  - the first call on each device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before capturing a stream into a graph.  cudaDeviceReset
//    destroys the module copy the cached address points into: after a reset
//    this entry point must not be called again in the same process;
//  - a probe that runs past its bound (the table holds at least twice the
//    rows, so a probe finds a free slot before that) is reported to the caller
//    by *count = -1 once the call's work has run, in place of the row count.
#include <mutex>

#include "vqnqs_internal.cuh"

namespace vq {

constexpr int kNoallocMaxRows = 1 << 18;
constexpr int kNoallocSlots = 1 << 19;
constexpr size_t kNoallocKeyBytes = (size_t)kNoallocSlots * sizeof(unsigned long long);
constexpr size_t kNoallocValBytes = (size_t)kNoallocSlots * sizeof(int);
constexpr size_t kNoallocBytes = kNoallocKeyBytes + kNoallocValBytes + 256;  // + status word

// 6 MiB + 256 B: hash keys, then hash values, then a status word.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The status word of this array is cleared by each call before its hash kernels
// run; afterwards a raised overflow bit turns the returned count into -1.
__global__ void k_noalloc_status_clear(int* status) { *status = 0; }
__global__ void k_noalloc_report(const int* __restrict__ status, int* __restrict__ count) {
    if (*status & VQNQS_DEV_HASH_OVERFLOW) *count = -1;
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
}  // namespace

}  // namespace vq

using namespace vq;

extern "C" int vqnqs_compress_rows_noalloc(int R, const int* uid, const int* code, int* new_id, int* rep_uid,
                                           int* rep_code, int* count, void* stream) {
    if (R < 0 || R > kNoallocMaxRows) return VQNQS_ERR_ARG;
    if (!count || (R > 0 && (!uid || !code || !new_id || !rep_uid || !rep_code))) return VQNQS_ERR_ARG;
    (void)cudaGetLastError();  // an error left by earlier, unrelated work is not this call's
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VQNQS_ERR_CUDA;
    void* base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_ptr[dev]) {  // once per device, with that device current
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VQNQS_ERR_CUDA;
            int n = 0;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
                return VQNQS_ERR_CUDA;
            g_sms[dev] = n;
            g_ptr[dev] = p;
        }
        base = g_ptr[dev];
        sms = g_sms[dev];
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(b);
    int* vals = reinterpret_cast<int*>(b + kNoallocKeyBytes);
    int* status = reinterpret_cast<int*>(b + kNoallocKeyBytes + kNoallocValBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_status_clear<<<1, 1, 0, st>>>(status);
    // the clear step zeroes the keys this call uses and *count
    cudaError_t e = launch_compress_pairs(R, uid, code, new_id, rep_uid, rep_code, count, keys, vals,
                                          compress_hash_bits(R), status, st, sms);
    if (e != cudaSuccess) return VQNQS_ERR_CUDA;
    k_noalloc_report<<<1, 1, 0, st>>>(status, count);
    return cudaGetLastError() == cudaSuccess ? VQNQS_OK : VQNQS_ERR_CUDA;
}
