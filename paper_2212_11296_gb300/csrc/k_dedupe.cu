// Compressed (I, V) representation of the hidden states (Sec. 3.2).
//
// After the quantizer of layer l, the input of every per-location operation of
// that layer is fixed by the pair (row id at layer l, codeword index): the
// residual stream x_l is a function of the row id and the quantized vector of
// the codeword.  Rows with equal pairs therefore share one new row id, and the
// per-location work runs once per id.  The table is an open-addressing hash
// (linear probing, load <= 1/2) over 64-bit keys; the thread whose CAS claims
// a slot takes a fresh id with atomicAdd and records the representative pair.
// A second pass looks every row's key up.  Probes are bounded by the table
// size; running past the bound sets VQNQS_DEV_HASH_OVERFLOW and leaves the row
// on id 0 instead of spinning.
//
// With reuse off, every row keeps its own id (the plain full recompute).
#include "vqnqs_internal.cuh"

namespace vq {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdULL;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ULL;
    z ^= z >> 33;
    return z;
}

__device__ __forceinline__ unsigned long long make_key(int uid, int code) {
    return ((((unsigned long long)(unsigned)uid) << 16) | (unsigned)code) + 1ULL;  // 0 = empty slot
}

__global__ void k_hash_clear(unsigned long long* __restrict__ keys, size_t H, int* __restrict__ counters,
                             int u_slot_next) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < H; i += (size_t)gridDim.x * blockDim.x)
        keys[i] = 0ULL;
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[u_slot_next] = 0;
}

__global__ void k_dedupe_insert(const int* __restrict__ uid_cur, const int* __restrict__ code,
                                int* __restrict__ counters, int u_slot_next, unsigned long long* __restrict__ keys,
                                int* __restrict__ vals, unsigned long long mask, int* __restrict__ rep_uid,
                                int* __restrict__ rep_code, int* __restrict__ status) {
    const int R = counters[CNT_R];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const int u = uid_cur[r], c = code[r];
        const unsigned long long key = make_key(u, c);
        unsigned long long h = mix64(key) & mask;
        bool done = false;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            unsigned long long prev = atomicCAS(&keys[h], 0ULL, key);
            if (prev == 0ULL) {
                const int id = atomicAdd(&counters[u_slot_next], 1);
                vals[h] = id;
                rep_uid[id] = u;
                rep_code[id] = c;
                done = true;
                break;
            }
            if (prev == key) { done = true; break; }
            h = (h + 1) & mask;
        }
        if (!done) atomicOr(status, VQNQS_DEV_HASH_OVERFLOW);
    }
}

__global__ void k_dedupe_lookup(const int* __restrict__ uid_cur, const int* __restrict__ code,
                                const int* __restrict__ counters, const unsigned long long* __restrict__ keys,
                                const int* __restrict__ vals, unsigned long long mask, int* __restrict__ uid_next,
                                int* __restrict__ status) {
    const int R = counters[CNT_R];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const unsigned long long key = make_key(uid_cur[r], code[r]);
        unsigned long long h = mix64(key) & mask;
        int id = -1;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            unsigned long long k = keys[h];
            if (k == key) { id = vals[h]; break; }
            if (k == 0ULL) break;
            h = (h + 1) & mask;
        }
        if (id < 0) {
            atomicOr(status, VQNQS_DEV_HASH_OVERFLOW);
            id = 0;
        }
        uid_next[r] = id;
    }
}

__global__ void k_identity_keys(const int* __restrict__ uid_cur, const int* __restrict__ code,
                                int* __restrict__ counters, int u_slot_next, int* __restrict__ uid_next,
                                int* __restrict__ rep_uid, int* __restrict__ rep_code) {
    const int R = counters[CNT_R];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        uid_next[r] = r;
        rep_uid[r] = uid_cur[r];
        rep_code[r] = code[r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[u_slot_next] = R;
}

cudaError_t launch_dedupe(const int* uid_cur, const int* code, int* counters, int u_slot_next, int Rmax,
                          unsigned long long* keys, int* vals, int hash_bits, int* uid_next, int* rep_uid,
                          int* rep_code, int reuse, int* status, cudaStream_t st, int num_sms) {
    int grid = (Rmax + 255) / 256;
    if (grid > 8 * num_sms) grid = 8 * num_sms;
    if (grid < 1) grid = 1;
    if (!reuse) {
        k_identity_keys<<<grid, 256, 0, st>>>(uid_cur, code, counters, u_slot_next, uid_next, rep_uid, rep_code);
        return cudaGetLastError();
    }
    const size_t H = (size_t)1 << hash_bits;
    const unsigned long long mask = (unsigned long long)H - 1ULL;
    k_hash_clear<<<8 * num_sms, 256, 0, st>>>(keys, H, counters, u_slot_next);
    k_dedupe_insert<<<grid, 256, 0, st>>>(uid_cur, code, counters, u_slot_next, keys, vals, mask, rep_uid, rep_code,
                                          status);
    k_dedupe_lookup<<<grid, 256, 0, st>>>(uid_cur, code, counters, keys, vals, mask, uid_next, status);
    return cudaGetLastError();
}

}  // namespace vq
