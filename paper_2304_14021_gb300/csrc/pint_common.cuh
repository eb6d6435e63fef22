// pint_common.cuh - types and device building blocks shared by the libpint kernels.
//
// Layout conventions (all kernels):
//   U, r, s        [n][y][x] real, x fastest, n = 0..nt-1 (time levels 1..N_t)
//   S (spectrum)   [k][y][x] complex, k = 0..nt/2 (half spectrum of the real
//                  time signal; the other half is its complex conjugate)
// Forward transforms use exp(-2 pi i jk/N) and are unnormalized; every
// normalization sits in the inverse path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace pint {

// Programmatic dependent launch (sm_90 and later).  A kernel started with
// launch_pdl may begin while its predecessor in the stream is still draining
// (its launch and the predecessor's tail overlap); it calls pdl_wait() before
// it reads or writes anything, which returns once the predecessor has
// completed and its memory is visible.  In a kernel launched the plain way
// pdl_wait() returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}


// Exact FP32 -> FP64 conversion by bit assembly on the integer pipes (the
// conversion instruction would run on the FP64 pipe).  Normal numbers rebias
// the exponent; zeros, subnormals (normalized here), infinities and NaNs are
// handled by the same integer operations.  For T = double it is the identity.
__device__ __forceinline__ double f32_to_f64_exact(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t sgn = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
    uint32_t hi, lo;
    if (e - 1u < 0xFEu) {            // normal
        hi = sgn | ((e + 896u) << 20) | (m >> 3);
        lo = m << 29;
    } else if (e == 0xFFu) {         // infinity / NaN
        hi = sgn | 0x7FF00000u | (m >> 3);
        lo = m << 29;
    } else if (m == 0u) {            // zero
        hi = sgn;
        lo = 0u;
    } else {                         // subnormal: m 2^-149 with the leading bit of m at position p
        const int p = 31 - __clz((int)m);
        const uint32_t mn = (m << (23 - p)) & 0x7FFFFFu;   // fraction bits after the leading one
        hi = sgn | ((uint32_t)(p + 874) << 20) | (mn >> 3);
        lo = mn << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double f32_to_f64_exact(double d) { return d; }
// FP64 -> FP32 by truncating the significand on the integer pipes (for norm
// partial sums only: no rounding, values outside the float range go to 0 or
// infinity); keeps the conversion instruction off the FP64 pipe.
__device__ __forceinline__ float f64_to_f32_trunc(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    const uint32_t sgn = hi & 0x80000000u;
    if (e <= 0) return __uint_as_float(sgn);
    if (e >= 255) return __uint_as_float(sgn | 0x7F800000u);
    return __uint_as_float(sgn | ((uint32_t)e << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

template <class T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <class T> using c_t = typename cplx_of<T>::type;

template <class C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

__host__ __device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <class C> __device__ __forceinline__ C operator+(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C operator-(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <class C> __device__ __forceinline__ C conjc(C a) { return mkc(a.x, -a.y); }
template <class C, class R> __device__ __forceinline__ C scalec(C a, R s) { return mkc(a.x * s, a.y * s); }
// a / b for complex b != 0
template <class C> __device__ __forceinline__ C cdiv(C a, C b) {
    using R = typename real_of<C>::type;
    R inv = R(1) / (b.x * b.x + b.y * b.y);
    return mkc((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
// multiply by exp(DIR * i pi/2): DIR=-1 -> -i, DIR=+1 -> +i
template <int DIR, class C> __device__ __forceinline__ C rot90(C a) {
    return DIR < 0 ? mkc(a.y, -a.x) : mkc(-a.y, a.x);
}

// ---------------------------------------------------------------------------
// Small DFTs in registers: X_k = sum_j v_j exp(DIR 2 pi i jk / R)
// ---------------------------------------------------------------------------
template <int DIR, class C> __device__ __forceinline__ void dft2(C* v) {
    C a = v[0];
    v[0] = a + v[1];
    v[1] = a - v[1];
}
template <int DIR, class C> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
    C a = v0 + v2, b = v0 - v2, c = v1 + v3, d = rot90<DIR>(v1 - v3);
    v0 = a + c;
    v2 = a - c;
    v1 = b + d;
    v3 = b - d;
}
template <int DIR, class C> __device__ __forceinline__ void dft4(C* v) { dft4<DIR>(v[0], v[1], v[2], v[3]); }
template <int DIR, class C> __device__ __forceinline__ void dft8(C* v) {
    using R = typename real_of<C>::type;
    const R s = R(0.70710678118654752440);
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<DIR>(e0, e1, e2, e3);
    dft4<DIR>(o0, o1, o2, o3);
    // twiddles exp(DIR 2 pi i k/8), k = 1, 2, 3
    C t1 = DIR < 0 ? mkc(s * (o1.x + o1.y), s * (o1.y - o1.x)) : mkc(s * (o1.x - o1.y), s * (o1.x + o1.y));
    C t2 = rot90<DIR>(o2);
    C t3 = DIR < 0 ? mkc(s * (o3.y - o3.x), -s * (o3.x + o3.y)) : mkc(-s * (o3.x + o3.y), s * (o3.x - o3.y));
    v[0] = e0 + o0;
    v[4] = e0 - o0;
    v[1] = e1 + t1;
    v[5] = e1 - t1;
    v[2] = e2 + t2;
    v[6] = e2 - t2;
    v[3] = e3 + t3;
    v[7] = e3 - t3;
}
template <int R, int DIR, class C> __device__ __forceinline__ void dftR(C* v) {
    if constexpr (R == 2) dft2<DIR>(v);
    else if constexpr (R == 4) dft4<DIR>(v);
    else dft8<DIR>(v);
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
// Radix of the next Stockham pass when M = log2(remaining length): 8 while
// possible, 4x4 for 16, then 4 or 2.
constexpr int next_radix(int M) { return (M >= 3 && M != 4) ? 8 : (M == 4 || M == 2) ? 4 : 2; }

// ---------------------------------------------------------------------------
// Stockham autosort FFT on sequences held in shared memory, executed by the
// whole CTA.  Element i of sequence b lives at buf[b*SSTR + i*ESTR].  Each
// pass reads all inputs of the thread's butterflies into registers, barriers,
// then writes the outputs, so it works in place.  tw[j] = exp(-2 pi i j/N).
// Task mapping keeps neighbouring threads on neighbouring addresses: for
// column layouts (ESTR > 1) the batch index is fastest, for rows the
// butterfly index.
// ---------------------------------------------------------------------------
// SW = 1 (contiguous rows, ESTR = 1): element i of a sequence is stored at
// i ^ ((i >> 4) & 15), i.e. each aligned group of 16 elements (one 128-byte
// bank row for complex64) is permuted by its group index.  Stride-R writes of
// the early passes then hit distinct banks; unit-stride accesses stay
// conflict-free (a fixed XOR within each group).
template <int SW> __device__ __forceinline__ int swz(int i) { return SW ? (i ^ ((i >> 4) & 15)) : i; }

// PERM (first pass only): the sequence to transform is the even/odd
// reordering v_m = x_{2m}, v_{N-1-m} = x_{2m+1} of the natural-order data in
// buf, read in place (element m of v sits at 2m for m < N/2, at 2N-1-2m
// above); that input is in natural (not swizzled) order.
// Twiddles: w^1 (and w^2 for radix 8) come from the table, the other powers
// from at most two complex products of those.
template <class C, int N, int R, int NS, int DIR, int NTH, int B, int ESTR, int SSTR, int SW = 0,
          bool PERM = false>
__device__ __forceinline__ void stockham_pass(C* buf, const C* __restrict__ tw) {
    constexpr int NB = N / R;              // butterflies per sequence
    constexpr int NTASK = NB * B;
    constexpr int TPT = (NTASK + NTH - 1) / NTH;
    constexpr bool COL = ESTR > 1;
    C v[TPT][R];
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        int t = tid + q * NTH;
        if (TPT * NTH == NTASK || t < NTASK) {
            int b = COL ? t % B : t / NB;
            int j = COL ? t / B : t % NB;
            const C* src = buf + b * SSTR;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = j + r * NB;
                const int pm = PERM ? (m < N / 2 ? 2 * m : 2 * N - 1 - 2 * m) : swz<SW>(m);
                v[q][r] = src[pm * ESTR];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        int t = tid + q * NTH;
        if (TPT * NTH == NTASK || t < NTASK) {
            int b = COL ? t % B : t / NB;
            int j = COL ? t / B : t % NB;
            if constexpr (NS > 1) {
                constexpr int STEP = N / (NS * R);
                const int jm = j % NS;
                C w[R];
                w[1] = tw[jm * STEP];
                if (DIR > 0) w[1] = conjc(w[1]);
                if constexpr (R == 4) {
                    w[2] = cmul(w[1], w[1]);
                    w[3] = cmul(w[2], w[1]);
                } else if constexpr (R == 8) {
                    w[2] = tw[2 * jm * STEP];
                    if (DIR > 0) w[2] = conjc(w[2]);
                    w[3] = cmul(w[2], w[1]);
                    w[4] = cmul(w[2], w[2]);
                    w[5] = cmul(w[4], w[1]);
                    w[6] = cmul(w[4], w[2]);
                    w[7] = cmul(w[4], w[3]);
                }
#pragma unroll
                for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], w[r]);
            }
            dftR<R, DIR>(v[q]);
            C* dst = buf + b * SSTR;
            int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; ++r) dst[swz<SW>(base + r * NS) * ESTR] = v[q][r];
        }
    }
    __syncthreads();
}

template <class C, int N, int NS, int M, int DIR, int NTH, int B, int ESTR, int SSTR, int SW, bool PERM = false>
__device__ __forceinline__ void fft_passes(C* buf, const C* __restrict__ tw) {
    if constexpr (M > 0) {
        constexpr int R = next_radix(M);
        stockham_pass<C, N, R, NS, DIR, NTH, B, ESTR, SSTR, SW, PERM>(buf, tw);
        fft_passes<C, N, NS * R, M - ilog2(R), DIR, NTH, B, ESTR, SSTR, SW, false>(buf, tw);
    }
}

// ---------------------------------------------------------------------------
// Warp-level Stockham FFT: one sequence of length N in shared memory
// transformed by one warp.  Element i is stored at swz<1>(i) ^ key (key < 16:
// a further fixed permutation inside each 16-element group).  The first pass
// may read the even/odd reordering of the stored sequence (PERM) and may read
// natural-order input (RSW false); every write is swizzled.  Lane l owns
// butterflies j = l + 32 q of every pass; passes are separated by __syncwarp
// only, so the warps of a CTA run independently.
// ---------------------------------------------------------------------------
template <class C, int N, int R, int NS, int DIR, bool PERM, bool RSW>
__device__ __forceinline__ void warp_pass(C* buf, const C* __restrict__ tw, int lane, int key) {
    constexpr int NB = N / R;
    constexpr int TPL = (NB + 31) / 32;
    C v[TPL][R];
#pragma unroll
    for (int q = 0; q < TPL; ++q) {
        const int j = lane + 32 * q;
        if (NB % 32 == 0 || j < NB) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = j + r * NB;
                const int idx = PERM ? (m < N / 2 ? 2 * m : 2 * N - 1 - 2 * m) : m;
                v[q][r] = buf[RSW ? (swz<1>(idx) ^ key) : idx];
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < TPL; ++q) {
        const int j = lane + 32 * q;
        if (NB % 32 == 0 || j < NB) {
            if constexpr (NS > 1) {
                constexpr int STEP = N / (NS * R);
                const int jm = j % NS;
                C w[R];
                w[1] = tw[jm * STEP];
                if (DIR > 0) w[1] = conjc(w[1]);
                if constexpr (R == 4) {
                    w[2] = cmul(w[1], w[1]);
                    w[3] = cmul(w[2], w[1]);
                } else if constexpr (R == 8) {
                    w[2] = tw[2 * jm * STEP];
                    if (DIR > 0) w[2] = conjc(w[2]);
                    w[3] = cmul(w[2], w[1]);
                    w[4] = cmul(w[2], w[2]);
                    w[5] = cmul(w[4], w[1]);
                    w[6] = cmul(w[4], w[2]);
                    w[7] = cmul(w[4], w[3]);
                }
#pragma unroll
                for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], w[r]);
            }
            dftR<R, DIR>(v[q]);
            const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[swz<1>(base + r * NS) ^ key] = v[q][r];
        }
    }
    __syncwarp();
}

template <class C, int N, int NS, int M, int DIR, bool PERM, bool RSW>
__device__ __forceinline__ void warp_passes(C* buf, const C* __restrict__ tw, int lane, int key) {
    if constexpr (M > 0) {
        constexpr int R = next_radix(M);
        warp_pass<C, N, R, NS, DIR, PERM, RSW>(buf, tw, lane, key);
        warp_passes<C, N, NS * R, M - ilog2(R), DIR, false, true>(buf, tw, lane, key);
    }
}

// In-place FFT of one sequence by the calling warp (all 32 lanes; data visible
// to the warp before the call; ends with __syncwarp).
template <class C, int N, int DIR, bool PERM = false, bool RSW = true>
__device__ __forceinline__ void warp_fft(C* buf, const C* __restrict__ tw, int lane, int key = 0) {
    warp_passes<C, N, 1, ilog2(N), DIR, PERM, RSW>(buf, tw, lane, key);
}

// In-place length-N FFT (N a power of two) of B sequences in shared memory.
// The caller must __syncthreads() before (data ready); the last pass ends
// with a barrier.  SW: swizzled row layout (see swz); the result is stored
// swizzled.  PERM: transform the even/odd reordering of the stored
// natural-order sequences (see stockham_pass).
template <class C, int N, int DIR, int NTH, int B, int ESTR, int SSTR, int SW = 0, bool PERM = false>
__device__ __forceinline__ void smem_fft(C* buf, const C* __restrict__ tw) {
    fft_passes<C, N, 1, ilog2(N), DIR, NTH, B, ESTR, SSTR, SW, PERM>(buf, tw);
}

// ---------------------------------------------------------------------------
// Device control block of one solve (one per handle).
// ---------------------------------------------------------------------------
enum : int { ST_RUNNING = 1 };

struct Ctl {
    int status;       // ST_RUNNING while iterating; then PINT_OK / PINT_ENOCONV / PINT_EDIVERGED
    int iter;         // index k of the residual being evaluated
    int max_iter;
    int pad;
    double tol;
    double bnorm;     // ||b||_2
    double rho0;      // rho of the first residual of the window
    double rho;       // last rho
    double jbar;      // mean(3u^2) of the current iterate (Cahn-Hilliard)
    double sum_r2;
    double sum_u2;
    double tol_update;  // > 0: also stop when ||delta||_2 / ||U||_2 <= tol_update
    double dnorm;       // ||delta||_2 / ||U||_2 of the last correction
    double hist[256];
    double dhist[256];  // dnorm per iteration (when the update-size test is on)
};

// Geometry and coefficients of one problem (by value into kernels).
// A(u) = c2 Lap^2 u + c1 Lap u + cN Lap(u^3)    (u_t + A(u) = 0)
struct Geo {
    int nx, ny, dim, bc, nt, nspace;
    double dt, inv_dt, ihx2, ihy2;   // 1/h^2 per axis
    double c2, c1, cN;
    double th;                       // theta of the theta-method (1 or 1/2)
    int expl;                        // 1: the c1 Laplacian term acts on u_{n-1} (Eyre splitting)
};

// Reduction helpers (deterministic: fixed shuffle tree, fixed warp order).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace pint
