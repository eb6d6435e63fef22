// k_dst.cu - the sine path of Step 2 (simply supported axes, the paper's
// boundary condition (ii), Sec. 5.1): the DST-I of every row or column of the
// half spectrum by a complex FFT of the odd extension, with the pointwise
// shifted division of Eq. 2.8 fused between the forward and inverse transform.
#include "../../include/pint.h"
#include "pint_common.cuh"
#include "pint_kernels.h"
#include "spatial.cuh"

namespace pint {

// ---------------------------------------------------------------------------
// Sine path (simply supported axis with n + 1 = M / 2 a power of two): the
// DST-I  X_p = sum_j x_j sin(pi (p+1)(j+1) / (n+1))  by one complex FFT of
// length M of the odd extension z = (0, x_0 .. x_{n-1}, 0, -x_{n-1} .. -x_0):
// Z_q = -2i sum_j x_j sin(pi q (j+1) / (n+1)), so X_p = (i/2) Z_{p+1}.  The
// DST-I is its own inverse up to the factor 2/(n+1).  A CTA transforms LB
// lines at a time: rows (axis 0, line b = k ny + y, stride 1) or columns
// (axis 1, line b = k nx + x, stride nx; the LB lines of a tile are adjacent
// columns, so every row of the tile is one coalesced segment).
//   FWD: X = DST x;  INV: x = 2/(n+1) DST X;  FDI: both, with the division.
// ---------------------------------------------------------------------------
template <class T, int M> struct DstCfg {
    static constexpr int NTH = 256;
    static constexpr int LB0 = (int)((48 * 1024) / (M * sizeof(c_t<T>)));
    static constexpr int LB = LB0 < 1 ? 1 : (LB0 > 16 ? 16 : LB0);
    static constexpr size_t SMEM = (size_t)LB * M * sizeof(c_t<T>);
    static constexpr int N = M / 2, NV = N - 1;
    static constexpr int PPT = (LB * NV + NTH - 1) / NTH;   // coefficients per thread (FDI)
};

template <class T, int M, int MODE, int AXIS>
__global__ void __launch_bounds__(256) k_dst(int nx, int ny, long nlines, c_t<T>* __restrict__ S, Tabs<T> tb,
                                             SolveCoef co, const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    using Cfg = DstCfg<T, M>;
    constexpr int N = Cfg::N, NV = Cfg::NV, LB = Cfg::LB, NTH = Cfg::NTH, PPT = Cfg::PPT;
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const C* tw = AXIS == 0 ? tb.dsx : tb.dsy;
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    const int tid = threadIdx.x;
    // element j of line l: rows contiguous; columns at stride nx inside their slice
    auto addr = [&](long l, int j) -> size_t {
        if (AXIS == 0) return (size_t)l * NV + j;
        const long k = l / nx, x = l % nx;
        return ((size_t)k * ny + j) * nx + x;
    };
    // element e of the tile's values: (line b, index j), j-major for columns
    auto split = [&](int e, int& b, int& j) {
        if (AXIS == 0) {
            b = e / NV;
            j = e % NV;
        } else {
            j = e / LB;
            b = e % LB;
        }
    };
    // odd extension of v (line b, index j) into buf
    auto put = [&](int b, int j, C v) {
        buf[b * M + j + 1] = v;
        buf[b * M + M - 1 - j] = mkc(-v.x, -v.y);
    };
    for (long l0 = (long)blockIdx.x * LB; l0 < nlines; l0 += (long)gridDim.x * LB) {
        for (int e = tid; e < LB * NV; e += NTH) {
            int b, j;
            split(e, b, j);
            put(b, j, l0 + b < nlines ? S[addr(l0 + b, j)] : mkc(T(0), T(0)));
        }
        for (int b = tid; b < LB; b += NTH) {
            buf[b * M] = mkc(T(0), T(0));
            buf[b * M + N] = mkc(T(0), T(0));
        }
        __syncthreads();
        smem_fft<C, M, -1, NTH, LB, 1, M>(buf, tw);
        if constexpr (MODE == MODE_FDI) {
            // X_p = (i/2) Z_{p+1}, divided by the shifted eigenvalue, then extended again
            C v[PPT];
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const int e = tid + q * NTH;
                if (e < LB * NV) {
                    int b, p;
                    split(e, b, p);
                    const C Z = buf[b * M + p + 1];
                    C X = mkc(T(-0.5) * Z.y, T(0.5) * Z.x);
                    const long l = l0 + b;
                    if (l < nlines) {
                        const int k = AXIS == 0 ? (int)(l / ny) : (int)(l / nx);
                        const T Lam = AXIS == 0 ? tb.lamx[p] : tb.lamx[l % nx] + tb.lamy[p];
                        X = cdiv(X, shift_den(tb, k, Lam, c2, c1));
                    }
                    v[q] = X;
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                const int e = tid + q * NTH;
                if (e < LB * NV) {
                    int b, p;
                    split(e, b, p);
                    put(b, p, v[q]);
                }
            }
            for (int b = tid; b < LB; b += NTH) {
                buf[b * M] = mkc(T(0), T(0));
                buf[b * M + N] = mkc(T(0), T(0));
            }
            __syncthreads();
            smem_fft<C, M, -1, NTH, LB, 1, M>(buf, tw);
        }
        // FWD: (i/2) Z_{j+1};  INV, FDI: 2/(n+1) (i/2) Z_{j+1} = (i/N) Z_{j+1}
        const T sc = MODE == MODE_FWD ? T(0.5) : T(1) / T(N);
        for (int e = tid; e < LB * NV; e += NTH) {
            int b, j;
            split(e, b, j);
            if (l0 + b < nlines) {
                const C Z = buf[b * M + j + 1];
                S[addr(l0 + b, j)] = mkc(-sc * Z.y, sc * Z.x);
            }
        }
        __syncthreads();   // buf is refilled by the next tile
    }
}

// Resident CTAs (SMs x CTAs per SM) of one sine-path kernel: set, with its
// shared-memory attribute, by configure_dst outside any stream capture.
template <class T, int M, int MODE, int AXIS> static int& dst_per() {
    static int v = 0;
    return v;
}
template <class T, int M, int MODE, int AXIS> static cudaError_t dst_configure_one(int nsm) {
    using Cfg = DstCfg<T, M>;
    cudaError_t e = cudaSuccess;
    if (Cfg::SMEM > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_dst<T, M, MODE, AXIS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)Cfg::SMEM)) != cudaSuccess)
        return e;
    int per = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dst<T, M, MODE, AXIS>, Cfg::NTH, Cfg::SMEM)) !=
        cudaSuccess)
        return e;
    dst_per<T, M, MODE, AXIS>() = (per < 1 ? 1 : per) * nsm;
    return cudaSuccess;
}
template <class T, int M, int MODE, int AXIS>
static cudaError_t dst_m(int nx, int ny, long nlines, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                         cudaStream_t st) {
    using Cfg = DstCfg<T, M>;
    const long cap = dst_per<T, M, MODE, AXIS>();
    if (cap < 1) return cudaErrorInitializationError;   // configure_dst has not run
    const long tiles = (nlines + Cfg::LB - 1) / Cfg::LB;
    const int grid = (int)(tiles < cap ? tiles : cap);
    k_dst<T, M, MODE, AXIS><<<grid, Cfg::NTH, Cfg::SMEM, st>>>(nx, ny, nlines, S, tb, co, ctl);
    return cudaSuccess;
}
#define PINT_DST_SIZES(D_) D_(8) D_(16) D_(32) D_(64) D_(128) D_(256) D_(512) D_(1024) D_(2048) D_(4096) D_(8192)

// DST path of one axis of n points (n + 1 = M / 2 a power of two, 8 <= M <= 8192).
template <class T, int MODE, int AXIS>
cudaError_t dst_axis(int n, int nx, int ny, long nlines, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                     cudaStream_t st) {
    switch (2 * (n + 1)) {
#define D_(M) case M: return dst_m<T, M, MODE, AXIS>(nx, ny, nlines, S, tb, co, ctl, st);
        PINT_DST_SIZES(D_)
#undef D_
        default: return cudaErrorInvalidValue;
    }
}
int dst_axis_supported(int n) { return n >= 3 && n <= 4095 && ((n + 1) & n) == 0; }

template <class T, int M> static cudaError_t configure_dst_m(int axis, int nsm) {
    cudaError_t e;
    if (axis == 1) return dst_configure_one<T, M, MODE_FDI, 1>(nsm);
    if ((e = dst_configure_one<T, M, MODE_FDI, 0>(nsm)) != cudaSuccess) return e;
    if ((e = dst_configure_one<T, M, MODE_FWD, 0>(nsm)) != cudaSuccess) return e;
    return dst_configure_one<T, M, MODE_INV, 0>(nsm);
}
cudaError_t configure_dst(int n, int axis, int f32) {
    int dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    switch (2 * (n + 1)) {
#define D_(M) case M: return f32 ? configure_dst_m<float, M>(axis, nsm) : configure_dst_m<double, M>(axis, nsm);
        PINT_DST_SIZES(D_)
#undef D_
        default: return cudaErrorInvalidValue;
    }
}

#define PINT_DST_INST(T)                                                                                      \
    template cudaError_t dst_axis<T, MODE_FDI, 0>(int, int, int, long, c_t<T>*, const Tabs<T>&, SolveCoef,     \
                                                  const Ctl*, cudaStream_t);                                    \
    template cudaError_t dst_axis<T, MODE_FWD, 0>(int, int, int, long, c_t<T>*, const Tabs<T>&, SolveCoef,     \
                                                  const Ctl*, cudaStream_t);                                    \
    template cudaError_t dst_axis<T, MODE_INV, 0>(int, int, int, long, c_t<T>*, const Tabs<T>&, SolveCoef,     \
                                                  const Ctl*, cudaStream_t);                                    \
    template cudaError_t dst_axis<T, MODE_FDI, 1>(int, int, int, long, c_t<T>*, const Tabs<T>&, SolveCoef,     \
                                                  const Ctl*, cudaStream_t);
PINT_DST_INST(float)
PINT_DST_INST(double)
#undef PINT_DST_INST

}  // namespace pint
