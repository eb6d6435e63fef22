// k_jacobian.cu - the space-varying averaged Jacobian of Eq. 4.12 (paper-
// literal PinT-I / PinT-II): its field J~(x) = mean over the time levels of
// 3 u_n(x)^2, the variable-coefficient spatial operator of Step 2 applied to
// every frequency slice of the spectrum,
//   M_k y = lambda_1k y + lambda_2k (c2 Lap^2 y + Lap((c1 - J~) y)) + lambda_3k Lap y,
// (PinT-I: c1 = 1, lambda_3k = 0; PinT-II: c1 = 0, lambda_3k = 1 - dt lambda_1k),
// and the complex vector kernels of the inner flexible GMRES that solves it.
#include "ff.cuh"
#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

// jt[p] = 3/nt sum_n u_n[p]^2 from the FP64 iterate (uff == nullptr) or the float-float one.
template <class T>
__global__ void k_jtilde(const double* __restrict__ U, const float2* __restrict__ uff, int nt, int nspace,
                         T* __restrict__ jt) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nspace; p += gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int n = 0; n < nt; ++n) {
            const double u = uff ? (double)uff[(size_t)n * nspace + p].x : U[(size_t)n * nspace + p];
            a = fma(u, u, a);
        }
        jt[p] = (T)(3.0 * a / nt);
    }
}

// Reflected index of a halo point (same boundary treatment as the residual):
// returns -1 for a zero ghost (simply supported), sets the sign.
__device__ __forceinline__ int refl_index(int g, int n, int bc, float& sgn) {
    if (bc == 1) return g < 0 ? -1 - g : (g >= n ? 2 * n - 1 - g : g);
    if (bc == 2) return g < 0 ? -g : (g >= n ? 2 * (n - 1) - g : g);
    if (g == -1 || g == n) return -1;
    if (g < -1) { sgn = -sgn; return -2 - g; }
    if (g > n) { sgn = -sgn; return 2 * n - g; }
    return g;
}

// One CTA: a 32 x 8 tile of one frequency slice k = blockIdx.z (1-D: 256 x 1).
template <class T, int DIM>
__global__ void __launch_bounds__(256) k_apply_M(Geo g, int nk, const c_t<T>* __restrict__ Y, c_t<T>* __restrict__ W,
                                                 const T* __restrict__ jt, Tabs<T> tb, T c2, T c1) {
    using C = c_t<T>;
    constexpr int TX = DIM == 2 ? 32 : 256, TY = DIM == 2 ? 8 : 1, HY = DIM == 2 ? 2 : 0;
    constexpr int SX = TX + 4, SY = TY + 2 * HY, LX = TX + 2, LY = TY + (DIM == 2 ? 2 : 0);
    __shared__ C sy[SY * SX];   // y
    __shared__ C sq[SY * SX];   // (c1 - J~) y
    __shared__ C sL[LY * LX];   // Lap y
    const int k = blockIdx.z;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const C* Yk = Y + (size_t)k * g.nspace;
    for (int e = threadIdx.x; e < SX * SY; e += TX * TY) {
        const int ix = e % SX, iy = e / SX;
        float sgn = 1.f;
        const int gx = refl_index(x0 - 2 + ix, g.nx, g.bc, sgn);
        const int gy = DIM == 2 ? refl_index(y0 - HY + iy, g.ny, g.bc, sgn) : 0;
        C v = mkc(T(0), T(0));
        T q = T(0);
        if (gx >= 0 && gx < g.nx && gy >= 0 && (DIM == 1 || gy < g.ny)) {
            const int idx = (DIM == 2 ? gy * g.nx : 0) + gx;
            v = scalec(Yk[idx], T(sgn));
            q = c1 - jt[idx];
        }
        sy[e] = v;
        sq[e] = scalec(v, q);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LX * LY; e += TX * TY) {
        const int ix = e % LX, iy = e / LX;
        const int c = (DIM == 2 ? (iy + 1) * SX : 0) + ix + 1;
        C v = scalec(sy[c - 1] + sy[c + 1] - scalec(sy[c], T(2)), T(g.ihx2));
        if (DIM == 2) v = v + scalec(sy[c - SX] + sy[c + SX] - scalec(sy[c], T(2)), T(g.ihy2));
        sL[e] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= g.nx || (DIM == 2 && gy >= g.ny)) return;
    const int cl = (DIM == 2 ? (ty + 1) * LX : 0) + tx + 1;
    const int cu = (ty + HY) * SX + tx + 2;
    const C L = sL[cl];
    C L2 = scalec(sL[cl - 1] + sL[cl + 1] - scalec(L, T(2)), T(g.ihx2));
    if (DIM == 2) L2 = L2 + scalec(sL[cl - LX] + sL[cl + LX] - scalec(L, T(2)), T(g.ihy2));
    C Lq = scalec(sq[cu - 1] + sq[cu + 1] - scalec(sq[cu], T(2)), T(g.ihx2));
    if (DIM == 2) Lq = Lq + scalec(sq[cu - SX] + sq[cu + SX] - scalec(sq[cu], T(2)), T(g.ihy2));
    const C op = scalec(L2, c2) + Lq;                       // c2 Lap^2 y + Lap((c1 - J~) y)
    const C l1 = tb.lam1[k], l2 = tb.lam2[k];
    C w = cmul(l1, sy[cu]) + cmul(l2, op);
    if (tb.dte != T(0)) w = w + cmul(mkc(T(1) - tb.dte * l1.x, -tb.dte * l1.y), L);   // lambda_3k Lap y
    W[(size_t)k * g.nspace + (DIM == 2 ? gy * g.nx : 0) + gx] = w;
}

constexpr int kCDotThreads = 256;
constexpr int kGroup = 4;   // vectors handled per launch (register accumulators)

// partials[(b * ldp + i0 + i) * 2 + {0,1}] = CTA b's part of <v_i, w> = sum conj(v_i) w (FP64), i < G.
template <class T, int G>
__global__ void __launch_bounds__(kCDotThreads) k_cmulti_dot(const c_t<T>* __restrict__ w, const c_t<T>* __restrict__ V,
                                                            size_t ld, size_t n, int ldp, int i0,
                                                            double* __restrict__ partials) {
    __shared__ double red[kCDotThreads / 32][G][2];
    double re[G], im[G];
#pragma unroll
    for (int i = 0; i < G; ++i) re[i] = im[i] = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double wr = w[e].x, wi = w[e].y;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const c_t<T> v = V[i * ld + e];
            re[i] = fma((double)v.x, wr, fma((double)v.y, wi, re[i]));
            im[i] = fma((double)v.x, wi, fma(-(double)v.y, wr, im[i]));
        }
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int i = 0; i < G; ++i) {
        const double a = warp_sum(re[i]), b = warp_sum(im[i]);
        if (lane == 0) { red[warp][i][0] = a; red[warp][i][1] = b; }
    }
    __syncthreads();
    if (threadIdx.x < G) {
        const int i = threadIdx.x;
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kCDotThreads / 32; ++q) { a += red[q][i][0]; b += red[q][i][1]; }
        partials[((size_t)blockIdx.x * ldp + i0 + i) * 2] = a;
        partials[((size_t)blockIdx.x * ldp + i0 + i) * 2 + 1] = b;
    }
}

// w += sum_i c_i v_i, i < G, complex coefficients c (FP64 pairs on the device).
template <class T, int G>
__global__ void k_cmulti_axpy(c_t<T>* __restrict__ w, const c_t<T>* __restrict__ V, size_t ld,
                              const double* __restrict__ c, size_t n) {
    double cr[G], ci[G];
#pragma unroll
    for (int i = 0; i < G; ++i) { cr[i] = c[2 * i]; ci[i] = c[2 * i + 1]; }
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        double xr = w[e].x, xi = w[e].y;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const c_t<T> v = V[i * ld + e];
            xr += cr[i] * v.x - ci[i] * v.y;
            xi += cr[i] * v.y + ci[i] * v.x;
        }
        w[e] = mkc((T)xr, (T)xi);
    }
}

// z = a x + b y (real scalars; y may be nullptr)
template <class T>
__global__ void k_caxpby(c_t<T>* __restrict__ z, T a, const c_t<T>* __restrict__ x, T b, const c_t<T>* __restrict__ y,
                         size_t n) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        c_t<T> v = scalec(x[e], a);
        if (y) v = v + scalec(y[e], b);
        z[e] = v;
    }
}

static int grid_n(size_t n) {
    const size_t b = (n + 255) / 256;
    return (int)(b > 2 * 152 * 4 ? 2 * 152 * 4 : (b < 1 ? 1 : b));
}
int cdot_blocks(size_t n) { return grid_n(n); }

template <class T>
void launch_jtilde(const double* U, const float2* uff, int nt, int nspace, T* jt, cudaStream_t st) {
    k_jtilde<T><<<grid_n(nspace), 256, 0, st>>>(U, uff, nt, nspace, jt);
}
template <class T>
void launch_apply_M(const Geo& g, int nk, const c_t<T>* Y, c_t<T>* W, const T* jt, const Tabs<T>& tb, double c2,
                    double c1, cudaStream_t st) {
    if (g.dim == 2) {
        dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, nk);
        k_apply_M<T, 2><<<grid, 256, 0, st>>>(g, nk, Y, W, jt, tb, (T)c2, (T)c1);
    } else {
        dim3 grid((g.nx + 255) / 256, 1, nk);
        k_apply_M<T, 1><<<grid, 256, 0, st>>>(g, nk, Y, W, jt, tb, (T)c2, (T)c1);
    }
}
// Groups of up to kGroup vectors per launch, register accumulators.  Note:
// w may itself be one of the v_i (the axpy reads w[e] before writing it).
template <class T>
void launch_cmulti_dot(const c_t<T>* w, const c_t<T>* V, size_t ld, int nv, size_t n, double* partials,
                       cudaStream_t st) {
    const int nb = grid_n(n);
    for (int i0 = 0; i0 < nv; i0 += kGroup) {
        const c_t<T>* Vi = V + (size_t)i0 * ld;
        switch (nv - i0 >= kGroup ? kGroup : nv - i0) {
            case 1: k_cmulti_dot<T, 1><<<nb, kCDotThreads, 0, st>>>(w, Vi, ld, n, nv, i0, partials); break;
            case 2: k_cmulti_dot<T, 2><<<nb, kCDotThreads, 0, st>>>(w, Vi, ld, n, nv, i0, partials); break;
            case 3: k_cmulti_dot<T, 3><<<nb, kCDotThreads, 0, st>>>(w, Vi, ld, n, nv, i0, partials); break;
            default: k_cmulti_dot<T, 4><<<nb, kCDotThreads, 0, st>>>(w, Vi, ld, n, nv, i0, partials); break;
        }
    }
}
template <class T>
void launch_cmulti_axpy(c_t<T>* w, const c_t<T>* V, size_t ld, int nv, const double* c, size_t n, cudaStream_t st) {
    const int nb = grid_n(n);
    for (int i0 = 0; i0 < nv; i0 += kGroup) {
        const c_t<T>* Vi = V + (size_t)i0 * ld;
        const double* ci = c + 2 * i0;
        switch (nv - i0 >= kGroup ? kGroup : nv - i0) {
            case 1: k_cmulti_axpy<T, 1><<<nb, 256, 0, st>>>(w, Vi, ld, ci, n); break;
            case 2: k_cmulti_axpy<T, 2><<<nb, 256, 0, st>>>(w, Vi, ld, ci, n); break;
            case 3: k_cmulti_axpy<T, 3><<<nb, 256, 0, st>>>(w, Vi, ld, ci, n); break;
            default: k_cmulti_axpy<T, 4><<<nb, 256, 0, st>>>(w, Vi, ld, ci, n); break;
        }
    }
}
template <class T>
void launch_caxpby(c_t<T>* z, double a, const c_t<T>* x, double b, const c_t<T>* y, size_t n, cudaStream_t st) {
    k_caxpby<T><<<grid_n(n), 256, 0, st>>>(z, (T)a, x, (T)b, y, n);
}

#define PINT_INST(T)                                                                                              \
    template void launch_jtilde<T>(const double*, const float2*, int, int, T*, cudaStream_t);                      \
    template void launch_apply_M<T>(const Geo&, int, const c_t<T>*, c_t<T>*, const T*, const Tabs<T>&, double,    \
                                    double, cudaStream_t);                                                        \
    template void launch_cmulti_dot<T>(const c_t<T>*, const c_t<T>*, size_t, int, size_t, double*, cudaStream_t); \
    template void launch_cmulti_axpy<T>(c_t<T>*, const c_t<T>*, size_t, int, const double*, size_t, cudaStream_t); \
    template void launch_caxpby<T>(c_t<T>*, double, const c_t<T>*, double, const c_t<T>*, size_t, cudaStream_t);
PINT_INST(float)
PINT_INST(double)
#undef PINT_INST

}  // namespace pint
