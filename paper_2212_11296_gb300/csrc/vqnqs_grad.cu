// Small kernels of the gradient entry point: per-sample seeds of the energy
// gradient (Sec. 2) and the codebook term of the straight-through backward.
#include "vqnqs_internal.cuh"

namespace vq {

// seeds[b] = 2 (e[b] - mean e) / B, mean in FP64
__global__ void k_seeds_from_eloc(const float* __restrict__ e, int B, float* __restrict__ seeds) {
    __shared__ double s_w[32];
    __shared__ double s_mean;
    double a = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) a += (double)e[i];
    a = warp_sum_d(a);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s_w[i];
        s_mean = t / B;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < B; i += blockDim.x) seeds[i] = (float)(2.0 * ((double)e[i] - s_mean) / B);
}

// out_z[j][t] -= csum_z[j] * W[j][t]
__global__ void k_sub_scaled_rows(float* __restrict__ out, const float* __restrict__ csum, const float* __restrict__ W,
                                  int K, int d, int groups, long long stride) {
    const long long n = (long long)groups * K * d;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / ((long long)K * d));
        const int rem = (int)(i - (long long)z * K * d);
        const int j = rem / d;
        out[z * stride + rem] -= csum[(size_t)z * K + j] * W[rem];
    }
}

cudaError_t launch_seeds_from_eloc(const float* e_loc, int B, float* seeds, cudaStream_t st) {
    k_seeds_from_eloc<<<1, 1024, 0, st>>>(e_loc, B, seeds);
    return cudaGetLastError();
}
cudaError_t launch_sub_scaled_rows(float* out, const float* csum, const float* W, int K, int d, int groups,
                                   long long stride, cudaStream_t st, int cap) {
    long long n = (long long)groups * K * d;
    long long g = (n + 255) / 256;
    if (g > cap) g = cap;
    k_sub_scaled_rows<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(out, csum, W, K, d, groups, stride);
    return cudaGetLastError();
}

}  // namespace vq
