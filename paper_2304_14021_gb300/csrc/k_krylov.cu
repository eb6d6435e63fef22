// k_krylov.cu - vector kernels of the restarted flexible GMRES that can wrap
// the preconditioner P_alpha^{-1} (outer Krylov acceleration of the PinT
// iteration for the linear equations): several dot products against one
// vector in one pass, several scaled subtractions in one pass, and scaling.
// All in FP64.  The dot products leave per-CTA partial sums that the host adds
// in a fixed order, so results do not depend on scheduling.
#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

constexpr int kDotThreads = 256;

// partials[b * nv + i] = sum over CTA b's elements of w . v_i, i < nv (v_i = V + i * ld).
__global__ void __launch_bounds__(kDotThreads) k_multi_dot(const double* __restrict__ w, const double* __restrict__ V,
                                                          size_t ld, int nv, size_t n, double* __restrict__ partials) {
    __shared__ double red[kDotThreads / 32][kMaxKrylov + 1];
    double acc[kMaxKrylov + 1];
    for (int i = 0; i < nv; ++i) acc[i] = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double x = w[e];
        for (int i = 0; i < nv; ++i) acc[i] = fma(x, V[i * ld + e], acc[i]);
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int i = 0; i < nv; ++i) {
        const double s = warp_sum(acc[i]);
        if (lane == 0) red[warp][i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < kDotThreads / 32; ++q) s += red[q][i];
        partials[(size_t)blockIdx.x * nv + i] = s;
    }
}

// w += sum_i c_i v_i, i < nv (coefficients on the device).
__global__ void k_multi_axpy(double* __restrict__ w, const double* __restrict__ V, size_t ld, int nv,
                             const double* __restrict__ c, size_t n) {
    __shared__ double cs[kMaxKrylov + 1];
    for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = c[i];
    __syncthreads();
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double x = w[e];
        for (int i = 0; i < nv; ++i) x = fma(cs[i], V[i * ld + e], x);
        w[e] = x;
    }
}

// y = a * x
__global__ void k_scale_copy(double* __restrict__ y, const double* __restrict__ x, double a, size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = a * x[e];
}

int krylov_dot_blocks(size_t n) {
    const size_t b = (n + kDotThreads - 1) / kDotThreads;
    return (int)(b > 2 * 152 * 4 ? 2 * 152 * 4 : (b < 1 ? 1 : b));
}

void launch_multi_dot(const double* w, const double* V, size_t ld, int nv, size_t n, double* partials,
                      cudaStream_t st) {
    k_multi_dot<<<krylov_dot_blocks(n), kDotThreads, 0, st>>>(w, V, ld, nv, n, partials);
}
void launch_multi_axpy(double* w, const double* V, size_t ld, int nv, const double* c, size_t n, cudaStream_t st) {
    k_multi_axpy<<<krylov_dot_blocks(n), 256, 0, st>>>(w, V, ld, nv, c, n);
}
void launch_scale_copy(double* y, const double* x, double a, size_t n, cudaStream_t st) {
    k_scale_copy<<<krylov_dot_blocks(n), 256, 0, st>>>(y, x, a, n);
}

}  // namespace pint
