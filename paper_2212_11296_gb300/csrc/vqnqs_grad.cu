// Small kernels of the gradient entry points: per-sample seeds of the energy
// gradient (Sec. 2), the per-rank partial sums of a sharded energy gradient and
// their combination, and the codebook term of the straight-through backward.
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

// The per-rank partial sums of the sharded energy gradient: the two FP32 weighted
// gradient sums widened to FP64, then sum E, sum E^2 and the sample count.
__global__ void k_grad_partials(const float* __restrict__ s_eo, const float* __restrict__ s_o, long long P,
                                double* __restrict__ out) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x) {
        out[k] = (double)s_eo[k];
        out[P + k] = (double)s_o[k];
    }
}
__global__ void k_eloc_sums(const float* __restrict__ e, int B, double* __restrict__ out3) {
    __shared__ double s_w[2][32];
    double a = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) {
        const double x = (double)e[i];
        a += x;
        q += x * x;
    }
    a = warp_sum_d(a);
    q = warp_sum_d(q);
    if ((threadIdx.x & 31) == 0) { s_w[0][threadIdx.x >> 5] = a; s_w[1][threadIdx.x >> 5] = q; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tq = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { ta += s_w[0][i]; tq += s_w[1][i]; }
        out3[0] = ta;
        out3[1] = tq;
        out3[2] = (double)B;
    }
}

// grad[k] = 2 (sum E O_k - Ebar sum O_k) / n with Ebar = sum E / n: the energy gradient
// 2 mean[(E - Ebar) O_k] of every rank's samples, from the summed partials (Sec. 2);
// mean_var = (Ebar, sum E^2 / n - Ebar^2).  n = 0 gives zeros.
__global__ void k_energy_grad_combine(const double* __restrict__ part, long long P, float* __restrict__ grad,
                                      double* __restrict__ mean_var) {
    const double n = part[2 * P + 2];
    const double mean = n > 0.0 ? part[2 * P] / n : 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < P; k += (long long)gridDim.x * blockDim.x)
        grad[k] = n > 0.0 ? (float)(2.0 * (part[k] - mean * part[P + k]) / n) : 0.f;
    if (mean_var && blockIdx.x == 0 && threadIdx.x == 0) {
        mean_var[0] = mean;
        mean_var[1] = n > 0.0 ? part[2 * P + 1] / n - mean * mean : 0.0;
    }
}

cudaError_t launch_grad_partials(const float* s_eo, const float* s_o, long long P, const float* e_loc, int B,
                                 double* out, cudaStream_t st, int cap) {
    long long g = (P + 255) / 256;
    if (g > cap) g = cap;
    k_grad_partials<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(s_eo, s_o, P, out);
    k_eloc_sums<<<1, 1024, 0, st>>>(e_loc, B, out + 2 * P);
    return cudaGetLastError();
}
cudaError_t launch_energy_grad_combine(const double* part, long long P, float* grad, double* mean_var, cudaStream_t st,
                                       int cap) {
    long long g = (P + 255) / 256;
    if (g > cap) g = cap;
    k_energy_grad_combine<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(part, P, grad, mean_var);
    return cudaGetLastError();
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
