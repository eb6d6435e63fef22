// k_spatial.cu - Step 2 of the diagonalized solve (Eq. 2.8; Eq. 4.14 for
// Cahn-Hilliard): for every time frequency k the shifted spatial system
//     (lambda_1k I + lambda_2k A) S2[k] = S1[k]
// becomes a pointwise division in the eigenbasis of the spatial Laplacian:
//     S^[k,p] / (lambda_1k + lambda_2k mu(Lam_p)),   mu(L) = c2 L^2 + c1 L,
// where Lam_p is the eigenvalue of Delta_h (2-D: Lam_x + Lam_y).
//
// Two transform paths per axis:
//  * cosine (cell-centred Neumann, n a power of two): DCT-II by one complex
//    FFT of length n (even/odd reordering + post-twiddle; Makhoul 1980).  For
//    complex data (the real and imaginary parts are transformed independently)
//    X_p = (w_p V_p + conj(w_p) V_{n-p}) / 2 with w_p = exp(-i pi p / 2n), and
//    its inverse V_p = conj(w_p) (X_p - i X_{n-p}); both pair p with n - p.
//  * dense (simply supported DST-I, or any n <= 1024): X = F x, x = F^{-1} X
//    with the basis matrices held in device tables.
// 1-D: one fused pass (transform, divide, inverse) per row.  2-D: x-forward
// over rows, fused y pass (transform, divide, inverse) over columns, x-inverse.
#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

enum { MODE_FWD = 0, MODE_INV = 1, MODE_FDI = 2 };

template <class T>
__device__ __forceinline__ c_t<T> shift_den(const Tabs<T>& tb, int k, T Lam, T c2, T c1) {
    const T mu = c2 * Lam * Lam + c1 * Lam;
    const c_t<T> l1 = tb.lam1[k], l2 = tb.lam2[k];
    return mkc(l1.x + l2.x * mu, l1.y + l2.y * mu);
}

template <class T>
__device__ __forceinline__ T solve_c1(SolveCoef co, const Ctl* ctl) {
    return co.ch ? T(1.0 - ctl->jbar) : T(co.c1);
}

// position of x_i in the even/odd reordered sequence v (v_j = x_2j, v_{n-1-j} = x_{2j+1})
__device__ __forceinline__ int dct_pos(int i, int n) { return (i & 1) ? n - 1 - (i >> 1) : (i >> 1); }

// DCT-II post-twiddle on the pair (p, q = n-p): V -> X.
template <class C>
__device__ __forceinline__ void dct_post(C Vp, C Vq, C wp, C wq, C& Xp, C& Xq) {
    using R = typename real_of<C>::type;
    const R h = R(0.5);
    Xp = scalec(cmul(wp, Vp) + cmul(conjc(wp), Vq), h);
    Xq = scalec(cmul(wq, Vq) + cmul(conjc(wq), Vp), h);
}
// inverse pre-twiddle on the pair: X -> V (p == 0 pairs with X_n = 0).
template <class C>
__device__ __forceinline__ void dct_pre(int p, C Xp, C Xq, C wp, C wq, C& Vp, C& Vq) {
    if (p == 0) {
        Vp = Xp;
        Vq = Xp;
        return;
    }
    Vp = cmul(conjc(wp), Xp - rot90<+1>(Xq));
    Vq = cmul(conjc(wq), Xq - rot90<+1>(Xp));
}

// ---------------------------------------------------------------------------
// Rows (x axis), cosine path.  ROWS rows of length N per CTA, contiguous.
// Row index gr = k * ny + y.
// ---------------------------------------------------------------------------
template <class T, int N> struct RowCfg {
    static constexpr int ROWS = N >= 2048 ? 1 : 2048 / N;
    static constexpr int NTH = 256;
    static constexpr int PADSH = 0;                                // padding measured no better (bank conflicts rose)
    static constexpr int RS = PADSH ? N + N / 8 : N;               // padded row stride
    static constexpr size_t SMEM = sizeof(c_t<T>) * (size_t)ROWS * RS;
};

template <class T, int N, int MODE>
__global__ void __launch_bounds__(256) k_rows_dct(int nrows, int ny, c_t<T>* __restrict__ S, Tabs<T> tb,
                                                  SolveCoef co, const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    constexpr int ROWS = RowCfg<T, N>::ROWS, NTH = RowCfg<T, N>::NTH, PS = RowCfg<T, N>::PADSH;
    constexpr int RS = RowCfg<T, N>::RS;
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x;
    const long r0 = (long)blockIdx.x * ROWS;
#pragma unroll 4
    for (int e = tid; e < ROWS * N; e += NTH) {
        const int b = e / N, i = e % N;
        const long gr = r0 + b;
        C x = gr < nrows ? S[gr * N + i] : mkc(T(0), T(0));
        buf[b * RS + padi<PS>(MODE == MODE_INV ? i : dct_pos(i, N))] = x;
    }
    __syncthreads();
    if (MODE != MODE_INV) smem_fft<C, N, -1, NTH, ROWS, 1, RS, PS>(buf, tb.twx);
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    for (int e = tid; e < ROWS * (N / 2 + 1); e += NTH) {
        const int b = e / (N / 2 + 1), p = e % (N / 2 + 1), q = (N - p) % N;
        C* row = buf + b * RS;
        const C wp = tb.wx[p], wq = tb.wx[q];
        C Xp, Xq;
        if (MODE == MODE_INV) {
            Xp = row[padi<PS>(p)];
            Xq = row[padi<PS>(q)];
        } else {
            dct_post(row[padi<PS>(p)], row[padi<PS>(q)], wp, wq, Xp, Xq);
        }
        if (MODE == MODE_FWD) {
            row[padi<PS>(p)] = Xp;
            row[padi<PS>(q)] = Xq;
            continue;
        }
        if (MODE == MODE_FDI) {
            const int k = (int)((r0 + b) / ny);
            if (r0 + b < nrows) {
                Xp = cdiv(Xp, shift_den(tb, k, tb.lamx[p], c2, c1));
                Xq = cdiv(Xq, shift_den(tb, k, tb.lamx[q], c2, c1));
            }
        }
        C Vp, Vq;
        dct_pre(p, Xp, Xq, wp, wq, Vp, Vq);
        row[padi<PS>(p)] = Vp;
        row[padi<PS>(q)] = Vq;
    }
    __syncthreads();
    if (MODE == MODE_FWD) {
#pragma unroll 4
        for (int e = tid; e < ROWS * N; e += NTH) {
            const int b = e / N, i = e % N;
            const long gr = r0 + b;
            if (gr < nrows) S[gr * N + i] = buf[b * RS + padi<PS>(i)];
        }
        return;
    }
    smem_fft<C, N, +1, NTH, ROWS, 1, RS, PS>(buf, tb.twx);
    const T inv = T(1) / T(N);
#pragma unroll 4
    for (int e = tid; e < ROWS * N; e += NTH) {
        const int b = e / N, i = e % N;
        const long gr = r0 + b;
        if (gr < nrows) S[gr * N + i] = scalec(buf[b * RS + padi<PS>(dct_pos(i, N))], inv);
    }
}

// ---------------------------------------------------------------------------
// Columns (y axis), cosine path, fused forward/divide/inverse.  CTA = one
// frequency k and CW consecutive x columns; buf[y][c].
// ---------------------------------------------------------------------------
template <class T, int N> struct ColCfg {
    // 16 complex columns = 128 B (FP32) / 256 B (FP64) per row: coalesced, and
    // small enough for several CTAs per SM.
    static constexpr int CW = sizeof(T) == 4 ? (N <= 512 ? 16 : 8) : (N <= 256 ? 16 : 8);
    // enough threads that each holds at most two radix-8 butterflies across a barrier
    static constexpr int NTH = N * CW >= 8192 ? 1024 : (N * CW >= 2048 ? 512 : 256);
    static constexpr size_t SMEM = sizeof(c_t<T>) * (size_t)N * CW;
};

template <class T, int N>
__global__ void __launch_bounds__(ColCfg<T, N>::NTH)
    k_cols_dct_fdi(int nx, c_t<T>* __restrict__ S, Tabs<T> tb, SolveCoef co, const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    constexpr int CW = ColCfg<T, N>::CW, NTH = ColCfg<T, N>::NTH;
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x;
    const int k = blockIdx.y;
    const int x0 = blockIdx.x * CW;
    C* slab = S + (size_t)k * N * nx;
    for (int e = tid; e < N * CW; e += NTH) {
        const int c = e % CW, y = e / CW;
        const int x = x0 + c;
        buf[dct_pos(y, N) * CW + c] = x < nx ? slab[(size_t)y * nx + x] : mkc(T(0), T(0));
    }
    __syncthreads();
    smem_fft<C, N, -1, NTH, CW, CW, 1>(buf, tb.twy);
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    for (int e = tid; e < (N / 2 + 1) * CW; e += NTH) {
        const int c = e % CW, p = e / CW, q = (N - p) % N;
        const int x = x0 + c;
        const C wp = tb.wy[p], wq = tb.wy[q];
        C Xp, Xq;
        dct_post(buf[p * CW + c], buf[q * CW + c], wp, wq, Xp, Xq);
        if (x < nx) {
            const T lx = tb.lamx[x];
            Xp = cdiv(Xp, shift_den(tb, k, lx + tb.lamy[p], c2, c1));
            Xq = cdiv(Xq, shift_den(tb, k, lx + tb.lamy[q], c2, c1));
        }
        C Vp, Vq;
        dct_pre(p, Xp, Xq, wp, wq, Vp, Vq);
        buf[p * CW + c] = Vp;
        buf[q * CW + c] = Vq;
    }
    __syncthreads();
    smem_fft<C, N, +1, NTH, CW, CW, 1>(buf, tb.twy);
    const T inv = T(1) / T(N);
    for (int e = tid; e < N * CW; e += NTH) {
        const int c = e % CW, y = e / CW;
        const int x = x0 + c;
        if (x < nx) slab[(size_t)y * nx + x] = scalec(buf[dct_pos(y, N) * CW + c], inv);
    }
}

// ---------------------------------------------------------------------------
// Dense path: one CTA per vector of length n (row: stride 1; column: stride nx).
//   FWD: X = F x;   INV: x = Finv X;   FDI: both with the division between.
// axis 0 = x (rows, vector b = k*ny + y), axis 1 = y (columns, b = k*nx + x).
// ---------------------------------------------------------------------------
template <class T, int MODE>
__global__ void __launch_bounds__(128) k_dense(int axis, int nx, int ny, int nvec, c_t<T>* __restrict__ S,
                                               Tabs<T> tb, SolveCoef co, const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = axis == 0 ? nx : ny;
    C* v = reinterpret_cast<C*>(smem_raw);
    C* w = v + n;
    const int b = blockIdx.x;
    if (b >= nvec) return;
    size_t base;
    int stride, k, xcol = 0;
    if (axis == 0) {
        base = (size_t)b * nx;
        stride = 1;
        k = b / ny;
    } else {
        k = b / nx;
        xcol = b % nx;
        base = (size_t)k * ny * nx + xcol;
        stride = nx;
    }
    const T* F = axis == 0 ? tb.fx : tb.fy;
    const T* Fi = axis == 0 ? tb.ix : tb.iy;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = S[base + (size_t)i * stride];
    __syncthreads();
    if (MODE != MODE_INV) {
        const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            T ax = 0, ay = 0;
            const T* Fr = F + (size_t)p * n;
            for (int j = 0; j < n; ++j) {
                const T f = Fr[j];
                ax += f * v[j].x;
                ay += f * v[j].y;
            }
            C X = mkc(ax, ay);
            if (MODE == MODE_FDI) {
                const T Lam = axis == 0 ? tb.lamx[p] : tb.lamx[xcol] + tb.lamy[p];
                X = cdiv(X, shift_den(tb, k, Lam, c2, c1));
            }
            w[p] = X;
        }
        __syncthreads();
        if (MODE == MODE_FWD) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) S[base + (size_t)i * stride] = w[i];
            return;
        }
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = v[i];
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        T ax = 0, ay = 0;
        const T* Ir = Fi + (size_t)j * n;
        for (int p = 0; p < n; ++p) {
            const T f = Ir[p];
            ax += f * w[p].x;
            ay += f * w[p].y;
        }
        S[base + (size_t)j * stride] = mkc(ax, ay);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <class T, int N>
static cudaError_t cfg_rows() {
    cudaError_t e;
    const int sm = (int)RowCfg<T, N>::SMEM;
    if ((e = cudaFuncSetAttribute(k_rows_dct<T, N, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_rows_dct<T, N, MODE_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    return cudaFuncSetAttribute(k_rows_dct<T, N, MODE_FDI>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}
template <class T, int N>
static cudaError_t cfg_cols() {
    return cudaFuncSetAttribute(k_cols_dct_fdi<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ColCfg<T, N>::SMEM);
}

template <class T>
cudaError_t configure_spatial_all() {
    cudaError_t e;
#define PINT_R(N) if ((e = cfg_rows<T, N>()) != cudaSuccess) return e;
#define PINT_C(N) if ((e = cfg_cols<T, N>()) != cudaSuccess) return e;
    PINT_R(2) PINT_R(4) PINT_R(8) PINT_R(16) PINT_R(32) PINT_R(64) PINT_R(128) PINT_R(256) PINT_R(512)
    PINT_R(1024) PINT_R(2048) PINT_R(4096)
    PINT_C(2) PINT_C(4) PINT_C(8) PINT_C(16) PINT_C(32) PINT_C(64) PINT_C(128) PINT_C(256) PINT_C(512)
    PINT_C(1024)
#undef PINT_R
#undef PINT_C
    const int dense_smem = (int)(2 * 1024 * sizeof(c_t<T>));
    if ((e = cudaFuncSetAttribute(k_dense<T, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, dense_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(k_dense<T, MODE_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, dense_smem)))
        return e;
    return cudaFuncSetAttribute(k_dense<T, MODE_FDI>, cudaFuncAttributeMaxDynamicSharedMemorySize, dense_smem);
}
template cudaError_t configure_spatial_all<float>();
template cudaError_t configure_spatial_all<double>();

template <class T, int N, int MODE>
static void rows_n(int nrows, int ny, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl, cudaStream_t st) {
    constexpr int ROWS = RowCfg<T, N>::ROWS;
    int grid = (nrows + ROWS - 1) / ROWS;
    k_rows_dct<T, N, MODE><<<grid, 256, RowCfg<T, N>::SMEM, st>>>(nrows, ny, S, tb, co, ctl);
}
template <class T, int MODE>
static cudaError_t rows_dct(int nx, int nrows, int ny, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                            cudaStream_t st) {
    switch (nx) {
#define R_(N) case N: rows_n<T, N, MODE>(nrows, ny, S, tb, co, ctl, st); break;
        R_(2) R_(4) R_(8) R_(16) R_(32) R_(64) R_(128) R_(256) R_(512) R_(1024) R_(2048) R_(4096)
#undef R_
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}
template <class T, int N>
static void cols_n(int nx, int nk, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl, cudaStream_t st) {
    constexpr int CW = ColCfg<T, N>::CW;
    dim3 grid((nx + CW - 1) / CW, nk);
    k_cols_dct_fdi<T, N><<<grid, ColCfg<T, N>::NTH, ColCfg<T, N>::SMEM, st>>>(nx, S, tb, co, ctl);
}
template <class T>
static cudaError_t cols_dct(int nx, int ny, int nk, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                            cudaStream_t st) {
    switch (ny) {
#define C_(N) case N: cols_n<T, N>(nx, nk, S, tb, co, ctl, st); break;
        C_(2) C_(4) C_(8) C_(16) C_(32) C_(64) C_(128) C_(256) C_(512) C_(1024)
#undef C_
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}
template <class T, int MODE>
static void dense(int axis, int nx, int ny, int nk, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                  cudaStream_t st) {
    const int n = axis == 0 ? nx : ny;
    const int nvec = axis == 0 ? nk * ny : nk * nx;
    k_dense<T, MODE><<<nvec, 128, 2 * n * sizeof(c_t<T>), st>>>(axis, nx, ny, nvec, S, tb, co, ctl);
}

template <class T>
cudaError_t launch_spatial_stage(int stage, const Geo& g, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, int fft_x,
                                 int fft_y, const Ctl* ctl, cudaStream_t st) {
    const int nk = g.nt / 2 + 1;
    const int ny = g.dim == 2 ? g.ny : 1;
    cudaError_t e = cudaSuccess;
    if (g.dim == 1) {
        if (stage != 0) return cudaSuccess;
        if (fft_x) e = rows_dct<T, MODE_FDI>(g.nx, nk, 1, S, tb, co, ctl, st);
        else dense<T, MODE_FDI>(0, g.nx, 1, nk, S, tb, co, ctl, st);
    } else if (stage == 0) {
        if (fft_x) e = rows_dct<T, MODE_FWD>(g.nx, nk * ny, ny, S, tb, co, ctl, st);
        else dense<T, MODE_FWD>(0, g.nx, ny, nk, S, tb, co, ctl, st);
    } else if (stage == 1) {
        if (fft_y) e = cols_dct<T>(g.nx, ny, nk, S, tb, co, ctl, st);
        else dense<T, MODE_FDI>(1, g.nx, ny, nk, S, tb, co, ctl, st);
    } else {
        if (fft_x) e = rows_dct<T, MODE_INV>(g.nx, nk * ny, ny, S, tb, co, ctl, st);
        else dense<T, MODE_INV>(0, g.nx, ny, nk, S, tb, co, ctl, st);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
template cudaError_t launch_spatial_stage<float>(int, const Geo&, float2*, const Tabs<float>&, SolveCoef, int, int,
                                                 const Ctl*, cudaStream_t);
template cudaError_t launch_spatial_stage<double>(int, const Geo&, double2*, const Tabs<double>&, SolveCoef, int, int,
                                                  const Ctl*, cudaStream_t);

}  // namespace pint
