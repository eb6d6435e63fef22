// k_timefft.cu - Steps 1 and 3 of the diagonalized solve (Eq. 2.8): the FFT
// along the time axis of the (already alpha-scaled) space-time block and its
// inverse followed by the Gamma_alpha^{-1} unscaling.
//
// The time signal at each spatial point is real, so two spatial points share
// one complex FFT (point a in the real part, point b in the imaginary part):
//   forward:  Z = FFT(s_a + i s_b),  S_a[k] = (Z_k + conj Z_{N-k})/2,
//             S_b[k] = (Z_k - conj Z_{N-k})/(2i),   k = 0..N/2;
//   inverse:  Z_k = S_a[k] + i S_b[k] over the full Hermitian spectrum,
//             z = IFFT(Z),  x_a = Re z, x_b = Im z.
// A CTA holds CW complex columns (2*CW consecutive spatial points) times all
// N_t time levels in shared memory: loads and stores are rows of CW
// consecutive values per time level / frequency, i.e. coalesced.
#include "../../include/pint.h"
#include "ff.cuh"
#include "pint_common.cuh"
#include "pint_kernels.h"
#include "tma.cuh"

namespace pint {


template <class T, int NT> struct TimeCfg {
    static constexpr int CW = sizeof(T) == 4 ? (NT <= 512 ? 32 : 16) : (NT <= 256 ? 32 : (NT == 512 ? 16 : 8));
    // enough threads that each holds at most two radix-8 butterflies across a barrier
    static constexpr int NTH = NT * CW >= 8192 ? 1024 : (NT * CW >= 2048 ? 512 : 256);
    static constexpr size_t SMEM = sizeof(c_t<T>) * ((size_t)NT * CW + NT);
};

template <class T, int NT>
__global__ void __launch_bounds__(TimeCfg<T, NT>::NTH)
    k_time_fwd(int nspace, const T* __restrict__ s, c_t<T>* __restrict__ S, const c_t<T>* __restrict__ twt,
               const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    constexpr int CW = TimeCfg<T, NT>::CW, NTH = TimeCfg<T, NT>::NTH;
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* z = reinterpret_cast<C*>(smem_raw);
    C* tw = z + NT * CW;
    const int tid = threadIdx.x;
    const long p0 = (long)blockIdx.x * 2 * CW;
    for (int i = tid; i < NT; i += NTH) tw[i] = twt[i];
    // complex64 transforms on rows of a multiple of 4 points: 128-bit loads of 4
    // residual values and 128-bit stores of 2 spectrum values per thread (the
    // groups of 4 are then all inside the grid or all outside)
    const bool vec = sizeof(T) == 4 && (nspace & 3) == 0;
    if constexpr (sizeof(T) == 4) {
        if (vec) {
            constexpr int CQ = CW / 4;
#pragma unroll 4
            for (int e = tid; e < NT * CQ; e += NTH) {
                const int c = (e % CQ) * 4, n = e / CQ;
                const long pa = p0 + c, pb = p0 + CW + c;
                const T* row = s + (size_t)n * nspace;
                const float4 a = pa < nspace ? __ldg(reinterpret_cast<const float4*>(row + pa)) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 b = pb < nspace ? __ldg(reinterpret_cast<const float4*>(row + pb)) : make_float4(0.f, 0.f, 0.f, 0.f);
                C* zz = z + n * CW + c;
                zz[0] = mkc(a.x, b.x);
                zz[1] = mkc(a.y, b.y);
                zz[2] = mkc(a.z, b.z);
                zz[3] = mkc(a.w, b.w);
            }
        }
    }
    if (!vec) {
#pragma unroll 8
        for (int e = tid; e < NT * CW; e += NTH) {
            const int c = e % CW, n = e / CW;
            const long pa = p0 + c, pb = p0 + CW + c;
            const T* row = s + (size_t)n * nspace;
            T a = pa < nspace ? row[pa] : T(0);
            T b = pb < nspace ? row[pb] : T(0);
            z[e] = mkc(a, b);
        }
    }
    __syncthreads();
    smem_fft<C, NT, -1, NTH, CW, CW, 1>(z, tw);
    const T half = T(0.5);
    if constexpr (sizeof(T) == 4) {
        if (vec) {
            constexpr int CH = CW / 2;
#pragma unroll 4
            for (int e = tid; e < (NT / 2 + 1) * CH; e += NTH) {
                const int c = (e % CH) * 2, k = e / CH, kr = (NT - k) % NT;
                const C zk0 = z[k * CW + c], zk1 = z[k * CW + c + 1];
                const C zr0 = z[kr * CW + c], zr1 = z[kr * CW + c + 1];
                const long pa = p0 + c, pb = p0 + CW + c;
                C* row = S + (size_t)k * nspace;
                if (pa < nspace)
                    *reinterpret_cast<float4*>(row + pa) = make_float4(half * (zk0.x + zr0.x), half * (zk0.y - zr0.y),
                                                                       half * (zk1.x + zr1.x), half * (zk1.y - zr1.y));
                if (pb < nspace)
                    *reinterpret_cast<float4*>(row + pb) = make_float4(half * (zk0.y + zr0.y), half * (zr0.x - zk0.x),
                                                                       half * (zk1.y + zr1.y), half * (zr1.x - zk1.x));
            }
            return;
        }
    }
#pragma unroll 4
    for (int e = tid; e < (NT / 2 + 1) * CW; e += NTH) {
        const int c = e % CW, k = e / CW;
        const C zk = z[k * CW + c];
        const C zr = z[((NT - k) % NT) * CW + c];
        const long pa = p0 + c, pb = p0 + CW + c;
        C* row = S + (size_t)k * nspace;
        if (pa < nspace) row[pa] = mkc(half * (zk.x + zr.x), half * (zk.y - zr.y));
        if (pb < nspace) row[pb] = mkc(half * (zk.y + zr.y), half * (zr.x - zk.x));
    }
}

// OUTK = 0: FP64 output (out = delta, or out += delta when accumulate);
// OUTK = 1: float-float iterate, outff += delta with delta = x * ginvf[n] in FP32.
template <class T, int NT, int OUTK>
__global__ void __launch_bounds__(TimeCfg<T, NT>::NTH)
    k_time_inv(int nspace, const c_t<T>* __restrict__ S, const c_t<T>* __restrict__ twt,
               const double* __restrict__ ginv, const float* __restrict__ ginvf, double* __restrict__ out,
               float2* __restrict__ outff, int accumulate, const Ctl* __restrict__ ctl,
               double* __restrict__ dpart) {
    using C = c_t<T>;
    constexpr int CW = TimeCfg<T, NT>::CW, NTH = TimeCfg<T, NT>::NTH;
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* z = reinterpret_cast<C*>(smem_raw);
    C* tw = z + NT * CW;
    const int tid = threadIdx.x;
    const long p0 = (long)blockIdx.x * 2 * CW;
    for (int i = tid; i < NT; i += NTH) tw[i] = twt[i];
    // complex64 spectrum and FP64 iterate on rows of an even number of points:
    // 128-bit accesses of two points per thread (pairs all inside or all outside)
    const bool vec = sizeof(T) == 4 && OUTK == 0 && (nspace & 1) == 0;
    if constexpr (sizeof(T) == 4 && OUTK == 0) {
        if (vec) {
            constexpr int CH = CW / 2;
#pragma unroll 4
            for (int e = tid; e < (NT / 2 + 1) * CH; e += NTH) {
                const int c = (e % CH) * 2, k = e / CH;
                const long pa = p0 + c, pb = p0 + CW + c;
                const C* row = S + (size_t)k * nspace;
                float4 A = pa < nspace ? __ldg(reinterpret_cast<const float4*>(row + pa)) : make_float4(0.f, 0.f, 0.f, 0.f);
                float4 B = pb < nspace ? __ldg(reinterpret_cast<const float4*>(row + pb)) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (k == 0 || k == NT / 2) { A.y = A.w = 0.f; B.y = B.w = 0.f; }  // real in exact arithmetic
                z[k * CW + c] = mkc(A.x - B.y, A.y + B.x);
                z[k * CW + c + 1] = mkc(A.z - B.w, A.w + B.z);
                if (k > 0 && k < NT / 2) {
                    z[(NT - k) * CW + c] = mkc(A.x + B.y, B.x - A.y);
                    z[(NT - k) * CW + c + 1] = mkc(A.z + B.w, B.z - A.w);
                }
            }
        }
    }
    if (!vec) {
#pragma unroll 4
        for (int e = tid; e < (NT / 2 + 1) * CW; e += NTH) {
            const int c = e % CW, k = e / CW;
            const long pa = p0 + c, pb = p0 + CW + c;
            const C* row = S + (size_t)k * nspace;
            C a = pa < nspace ? row[pa] : mkc(T(0), T(0));
            C b = pb < nspace ? row[pb] : mkc(T(0), T(0));
            if (k == 0 || k == NT / 2) { a.y = T(0); b.y = T(0); }  // real in exact arithmetic
            z[k * CW + c] = mkc(a.x - b.y, a.y + b.x);
            if (k > 0 && k < NT / 2) z[(NT - k) * CW + c] = mkc(a.x + b.y, b.x - a.y);
        }
    }
    if constexpr (sizeof(T) == 4 && OUTK == 0) {
        // the iterate's rows that the update reads, pulled into L2 while the
        // FFT runs: 4 lines of 128 B per level (the CTA's two 32-point
        // segments), one line per thread and pass; lines starting past the row
        // end are skipped
        if (vec && accumulate) {
            for (int i = tid; i < NT * 4; i += NTH) {
                const int n = i >> 2, q = i & 3;
                const long p = (q < 2 ? p0 : p0 + CW) + 16 * (q & 1);
                if (p < nspace) {
                    const double* a = out + (size_t)n * nspace + p;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
                }
            }
        }
    }
    __syncthreads();
    smem_fft<C, NT, +1, NTH, CW, CW, 1>(z, tw);
    // dpart != nullptr: per-CTA partial sums (sum delta^2, sum U_new^2) of the
    // correction and the updated iterate, for the update-size stopping test
    float d2 = 0.f, u2 = 0.f;
    const bool want = dpart != nullptr;
    if constexpr (sizeof(T) == 4 && OUTK == 0) {
        if (vec && accumulate) {
            // U + x gamma_n^{-1}/N_t, two points per 128-bit access
            constexpr int CH = CW / 2;
#pragma unroll 4
            for (int e = tid; e < NT * CH; e += NTH) {
                const int c = (e % CH) * 2, n = e / CH;
                const C v0 = z[n * CW + c], v1 = z[n * CW + c + 1];
                const long pa = p0 + c, pb = p0 + CW + c;
                const double gi = ginv[n];
                double* row = out + (size_t)n * nspace;
                if (pa < nspace) {
                    double2* q = reinterpret_cast<double2*>(row + pa);
                    const double2 u = __ldcs(q);
                    const double2 w = make_double2(fma(f32_to_f64_exact(v0.x), gi, u.x), fma(f32_to_f64_exact(v1.x), gi, u.y));
                    __stcs(q, w);
                    if (want) {
                        const float g32 = f64_to_f32_trunc(gi), da0 = v0.x * g32, da1 = v1.x * g32;
                        const float w0 = f64_to_f32_trunc(w.x), w1 = f64_to_f32_trunc(w.y);
                        d2 = fmaf(da1, da1, fmaf(da0, da0, d2));
                        u2 = fmaf(w1, w1, fmaf(w0, w0, u2));
                    }
                }
                if (pb < nspace) {
                    double2* q = reinterpret_cast<double2*>(row + pb);
                    const double2 u = __ldcs(q);
                    const double2 w = make_double2(fma(f32_to_f64_exact(v0.y), gi, u.x), fma(f32_to_f64_exact(v1.y), gi, u.y));
                    __stcs(q, w);
                    if (want) {
                        const float g32 = f64_to_f32_trunc(gi), db0 = v0.y * g32, db1 = v1.y * g32;
                        const float w0 = f64_to_f32_trunc(w.x), w1 = f64_to_f32_trunc(w.y);
                        d2 = fmaf(db1, db1, fmaf(db0, db0, d2));
                        u2 = fmaf(w1, w1, fmaf(w0, w0, u2));
                    }
                }
            }
        }
    }
#pragma unroll 4
    for (int e = tid; e < (vec && accumulate ? 0 : NT * CW); e += NTH) {
        const int c = e % CW, n = e / CW;
        const C v = z[e];
        const long pa = p0 + c, pb = p0 + CW + c;
        if constexpr (OUTK == 1) {
            const float gi = ginvf[n];
            float2* row = outff + (size_t)n * nspace;
            const float da = (float)v.x * gi, db = (float)v.y * gi;
            if (pa < nspace) {
                const float2 w = ff_add_f(row[pa], da);
                row[pa] = w;
                if (want) {
                    d2 = fmaf(da, da, d2);
                    u2 = fmaf(w.x, w.x, u2);
                }
            }
            if (pb < nspace) {
                const float2 w = ff_add_f(row[pb], db);
                row[pb] = w;
                if (want) {
                    d2 = fmaf(db, db, d2);
                    u2 = fmaf(w.x, w.x, u2);
                }
            }
            continue;
        }
        const double gi = ginv[n];
        double* row = out + (size_t)n * nspace;
        if (accumulate) {
            // FP64 unscaling and update in one FP64 fused multiply-add, U + x gamma_n^{-1}/N_t (one
            // rounding); the FP32 transform output enters exactly (conversion by bit assembly)
            const double xa = f32_to_f64_exact(v.x), xb = f32_to_f64_exact(v.y);
            if (pa < nspace) {
                const double w = fma(xa, gi, row[pa]);
                row[pa] = w;
                if (want) {
                    const float da = (float)v.x * f64_to_f32_trunc(gi), wf = f64_to_f32_trunc(w);
                    d2 = fmaf(da, da, d2);
                    u2 = fmaf(wf, wf, u2);
                }
            }
            if (pb < nspace) {
                const double w = fma(xb, gi, row[pb]);
                row[pb] = w;
                if (want) {
                    const float db = (float)v.y * f64_to_f32_trunc(gi), wf = f64_to_f32_trunc(w);
                    d2 = fmaf(db, db, d2);
                    u2 = fmaf(wf, wf, u2);
                }
            }
        } else {
            const double da = (double)v.x * gi, db = (double)v.y * gi;   // FP64 unscaling
            if (pa < nspace) row[pa] = da;
            if (pb < nspace) row[pb] = db;
        }
    }
    if (want) {  // deterministic block reduction (same tree every launch)
        __shared__ double red[2][32];
        double a = warp_sum((double)d2), b = warp_sum((double)u2);
        if (tid % 32 == 0) { red[0][tid / 32] = a; red[1][tid / 32] = b; }
        __syncthreads();
        if (tid == 0) {
            double A = 0.0, B = 0.0;
            for (int w = 0; w < NTH / 32; ++w) { A += red[0][w]; B += red[1][w]; }
            dpart[2 * blockIdx.x] = A;
            dpart[2 * blockIdx.x + 1] = B;
        }
    }
}

// Float-float update with the iterate tile prefetched: at entry one warp
// starts bulk asynchronous copies of the CTA's U rows (2*CW points x N_t
// levels) into shared memory, so they load while the spectrum is read and
// transformed; the update U += delta then reads U from shared memory.  Needs
// an even number of spatial points (16-byte aligned rows); N_t <= 512.
template <int NT> struct TimeTmaCfg {
    static constexpr int CW = 16;
    static constexpr int NTH = NT * CW >= 8192 ? 1024 : (NT * CW >= 2048 ? 512 : 256);
    static constexpr size_t TW_OFF = sizeof(float2) * (size_t)NT * CW;
    static constexpr size_t U_OFF = TW_OFF + sizeof(float2) * NT;
    static constexpr size_t BAR_OFF = U_OFF + sizeof(float2) * (size_t)NT * 2 * CW;
    static constexpr size_t SMEM = BAR_OFF + 16;
};

template <int NT>
__global__ void __launch_bounds__(TimeTmaCfg<NT>::NTH)
    k_time_inv_ff_tma(int nspace, const float2* __restrict__ S, const float2* __restrict__ twt,
                      const float* __restrict__ ginvf, float2* __restrict__ Uff, const Ctl* __restrict__ ctl,
                      double* __restrict__ dpart) {
    using C = float2;
    using Cfg = TimeTmaCfg<NT>;
    constexpr int CW = Cfg::CW, NTH = Cfg::NTH;
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* z = reinterpret_cast<C*>(smem_raw);
    C* tw = reinterpret_cast<C*>(smem_raw + Cfg::TW_OFF);
    float2* ub = reinterpret_cast<float2*>(smem_raw + Cfg::U_OFF);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + Cfg::BAR_OFF);
    const int tid = threadIdx.x;
    const long p0 = (long)blockIdx.x * 2 * CW;
    const int npts = (int)min((long)2 * CW, nspace - p0);   // even: nspace is even
    if (tid < 32) {
        if (tid == 0) {
            mbar_init(bar, 1);
            mbar_fence_init();
            mbar_arrive_expect_tx(bar, (uint32_t)(NT * npts * sizeof(float2)));
        }
        __syncwarp();
        for (int n = tid; n < NT; n += 32)
            bulk_g2s(ub + n * 2 * CW, Uff + (size_t)n * nspace + p0, (uint32_t)(npts * sizeof(float2)), bar);
    }
    for (int i = tid; i < NT; i += NTH) tw[i] = twt[i];
#pragma unroll 4
    for (int e = tid; e < (NT / 2 + 1) * CW; e += NTH) {
        const int c = e % CW, k = e / CW;
        const long pa = p0 + c, pb = p0 + CW + c;
        const C* row = S + (size_t)k * nspace;
        C a = pa < nspace ? row[pa] : mkc(0.f, 0.f);
        C b = pb < nspace ? row[pb] : mkc(0.f, 0.f);
        if (k == 0 || k == NT / 2) { a.y = 0.f; b.y = 0.f; }  // real in exact arithmetic
        z[k * CW + c] = mkc(a.x - b.y, a.y + b.x);
        if (k > 0 && k < NT / 2) z[(NT - k) * CW + c] = mkc(a.x + b.y, b.x - a.y);
    }
    __syncthreads();
    smem_fft<C, NT, +1, NTH, CW, CW, 1>(z, tw);
    if (!__syncthreads_and(mbar_wait_bounded(bar, 0))) {
        if (tid == 0) {
            atomicExch(const_cast<int*>(&ctl->status), (int)PINT_ECUDA);
            mbar_wait_bounded(bar, 0);   // let the copies in flight land before the CTA exits
        }
        __syncthreads();
        return;
    }
    float d2 = 0.f, u2 = 0.f;
    const bool want = dpart != nullptr;
#pragma unroll 4
    for (int e = tid; e < NT * CW; e += NTH) {
        const int c = e % CW, n = e / CW;
        const C v = z[e];
        const long pa = p0 + c, pb = p0 + CW + c;
        const float gi = ginvf[n];
        float2* row = Uff + (size_t)n * nspace;
        const float da = v.x * gi, db = v.y * gi;
        if (pa < nspace) {
            const float2 w = ff_add_f(ub[n * 2 * CW + c], da);
            row[pa] = w;
            if (want) {
                d2 = fmaf(da, da, d2);
                u2 = fmaf(w.x, w.x, u2);
            }
        }
        if (pb < nspace) {
            const float2 w = ff_add_f(ub[n * 2 * CW + CW + c], db);
            row[pb] = w;
            if (want) {
                d2 = fmaf(db, db, d2);
                u2 = fmaf(w.x, w.x, u2);
            }
        }
    }
    if (want) {  // deterministic block reduction (same tree every launch)
        __shared__ double red[2][32];
        double a = warp_sum((double)d2), b = warp_sum((double)u2);
        if (tid % 32 == 0) { red[0][tid / 32] = a; red[1][tid / 32] = b; }
        __syncthreads();
        if (tid == 0) {
            double A = 0.0, B = 0.0;
            for (int w = 0; w < NTH / 32; ++w) { A += red[0][w]; B += red[1][w]; }
            dpart[2 * blockIdx.x] = A;
            dpart[2 * blockIdx.x + 1] = B;
        }
    }
}

// ---------------------------------------------------------------------------
// Long time axes (1024 < N_t <= 2^20): multi-pass (four-step) FFT with
// N_t = f_0 f_1 ... f_{S-1}, S = 2 or 3 factors of 32..256.  The signal of the
// spatial point pair (2j, 2j+1) is the complex column
// z_j[n] = s[n][2j] + i s[n][2j+1] (the float2 / double2 view of a row).
// Digits: n = sum_s n_s istr_s with istr_s = prod_{j>s} f_j (n_0 most
// significant), k = sum_s k_s P_s with P_s = prod_{j<s} f_j (k_0 least
// significant).  In n k mod N only the products n_j k_i with i <= j survive, so
//   forward pass s transforms over n_s (stride istr_s) into k_s and multiplies
//   by e^{-2 pi i k_s P_s (sum_{j>s} n_j istr_j) / N};
// the storage slot of digit s holds n_s and then k_s, so after the last pass
// Z_k sits in row sum_s k_s istr_s (long_pos).  The inverse runs the passes
// from s = S-1 down to 0 with the opposite sign; the twiddle that pass s-1
// needs, e^{+2 pi i k_{s-1} P_{s-1} (sum_{j>=s} n_j istr_j) / N}, is applied at
// the end of pass s, and pass 0 writes x_n in natural order.  All passes work
// in place in a complex workspace of N_t x nspace/2; unpack forms the half
// spectrum of the real signals (pairs k, N-k) in natural order and pack
// rebuilds the full one.
// ---------------------------------------------------------------------------
LongPlan long_plan(int nt) {
    int l = 0;
    while ((1 << l) < nt) ++l;
    LongPlan pl{};
    pl.S = l > 16 ? 3 : 2;
    const int base = l / pl.S, rem = l % pl.S;
    // ascending factors: f_0, the output pass of the inverse, is the smallest
    for (int i = 0; i < pl.S; ++i) pl.f[i] = 1 << (base + (i >= pl.S - rem ? 1 : 0));
    for (int i = 0; i < pl.S; ++i) {
        pl.istr[i] = 1;
        for (int j = i + 1; j < pl.S; ++j) pl.istr[i] *= pl.f[j];
        pl.P[i] = 1;
        for (int j = 0; j < i; ++j) pl.P[i] *= pl.f[j];
    }
    auto lg = [](int v) { int l = 0; while ((1 << l) < v) ++l; return l; };
    for (int i = 0; i < pl.S; ++i) {
        pl.lf[i] = lg(pl.f[i]);
        pl.listr[i] = lg(pl.istr[i]);
        pl.lP[i] = lg(pl.P[i]);
    }
    return pl;
}

// One pass over digit s: CTA = (o, column block), o in [0, N/NL); element m of
// the transform sits in row (o / istr) NL istr + m istr + o % istr.
// DIR < 0 (forward), TW: multiply element m (= k_s) by
//   e^{-2 pi i (o % istr) m / (NL istr)}.
// DIR > 0 (inverse), TW: multiply element m (= n_s) by
//   e^{+2 pi i k_{s-1} (m istr + o % istr) / (fprev NL istr)},  k_{s-1} = (o / istr) % fprev.
template <class T, int NL, int DIR, bool TW>
__global__ void __launch_bounds__(TimeCfg<T, NL>::NTH)
    k_time_long_pass(int ncol, int istr, int fprev, int N, c_t<T>* __restrict__ z, const c_t<T>* __restrict__ twN,
                     const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    constexpr int CW = TimeCfg<T, NL>::CW, NTH = TimeCfg<T, NL>::NTH;
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + NL * CW;
    const int tid = threadIdx.x;
    const int o = blockIdx.y;
    const int j0 = blockIdx.x * CW;
    const int step = N / NL;
    const int ohi = o / istr, olo = o % istr;
    const size_t base = (size_t)ohi * NL * istr + olo;
    for (int i = tid; i < NL; i += NTH) tw[i] = twN[(size_t)i * step];
    for (int e = tid; e < NL * CW; e += NTH) {
        const int c = e % CW, m = e / CW;
        const size_t row = base + (size_t)m * istr;
        buf[e] = j0 + c < ncol ? z[row * ncol + j0 + c] : mkc(T(0), T(0));
    }
    __syncthreads();
    smem_fft<C, NL, DIR, NTH, CW, CW, 1>(buf, tw);
    for (int e = tid; e < NL * CW; e += NTH) {
        const int c = e % CW, m = e / CW;
        if (j0 + c >= ncol) continue;
        C v = buf[e];
        if (TW) {
            // both exponents stay below N: olo < istr, m < NL; k_{s-1} < fprev, m istr + olo < NL istr
            const int idx = DIR < 0 ? olo * m * (N / (NL * istr))
                                    : (ohi % fprev) * (m * istr + olo) * (N / (fprev * NL * istr));
            C w = twN[idx];
            if (DIR > 0) w = conjc(w);
            v = cmul(v, w);
        }
        const size_t row = base + (size_t)m * istr;
        z[row * ncol + j0 + c] = v;
    }
}

// Row-block mapping of the unpack / pack kernels: thread t of a CTA of
// kPackThreads takes column j = t % ncol of row kk = t / ncol of each group of
// RB = kPackThreads / ncol rows (ncol <= kPackThreads), or columns j, j +
// kPackThreads, ... of one row (ncol > kPackThreads); no division per element.
constexpr int kPackThreads = 256;

// S[k][2j], S[k][2j+1] (k = 0..N/2) from Z_k and Z_{N-k}.
template <class T>
__global__ void k_time_long_unpack(int N, LongPlan pl, int ncol, const c_t<T>* __restrict__ z, c_t<T>* __restrict__ S,
                                   const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    if (ctl && ctl->status != ST_RUNNING) return;
    const int K = N / 2 + 1;
    const T half = T(0.5);
    const int rb = ncol <= kPackThreads ? kPackThreads / ncol : 1;
    const int t = threadIdx.x, kk = ncol <= kPackThreads ? t / ncol : 0, j0 = ncol <= kPackThreads ? t % ncol : t;
    if (kk >= rb) return;
    for (int k = blockIdx.x * rb + kk; k < K; k += gridDim.x * rb) {
        const C* zrk = z + (size_t)long_pos(k, pl) * ncol;
        const C* zrr = z + (size_t)long_pos((N - k) & (N - 1), pl) * ncol;
        C* row = S + (size_t)k * 2 * ncol;
        for (int j = j0; j < ncol; j += kPackThreads) {
            const C zk = zrk[j], zr = zrr[j];
            row[2 * j] = mkc(half * (zk.x + zr.x), half * (zk.y - zr.y));
            row[2 * j + 1] = mkc(half * (zk.y + zr.y), half * (zr.x - zk.x));
        }
    }
}

// Z_k = S_a[k] + i S_b[k] over the full Hermitian spectrum, into the workspace rows of the last forward pass.
template <class T>
__global__ void k_time_long_pack(int N, LongPlan pl, int ncol, const c_t<T>* __restrict__ S, c_t<T>* __restrict__ z,
                                 const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    if (ctl && ctl->status != ST_RUNNING) return;
    const int rb = ncol <= kPackThreads ? kPackThreads / ncol : 1;
    const int t = threadIdx.x, kr = ncol <= kPackThreads ? t / ncol : 0, j0 = ncol <= kPackThreads ? t % ncol : t;
    if (kr >= rb) return;
    for (int k = blockIdx.x * rb + kr; k < N; k += gridDim.x * rb) {
        const int kk = k <= N / 2 ? k : N - k;
        const C* row = S + (size_t)kk * 2 * ncol;
        C* zr = z + (size_t)long_pos(k, pl) * ncol;
        for (int j = j0; j < ncol; j += kPackThreads) {
            C a = row[2 * j], b = row[2 * j + 1];
            if (kk == 0 || kk == N / 2) { a.y = T(0); b.y = T(0); }   // real in exact arithmetic
            if (k > N / 2) { a.y = -a.y; b.y = -b.y; }
            zr[j] = mkc(a.x - b.y, a.y + b.x);
        }
    }
}

// Inverse pass 0 (over k_0, rows m*istr0 + o, istr0 = N / f_0) and the output:
// x[n] at n = m*istr0 + o scaled by ginv[n] (which holds alpha^{-n/N}/N); OUTK
// as in k_time_inv.
template <class T, int NL, int OUTK>
__global__ void __launch_bounds__(TimeCfg<T, NL>::NTH)
    k_time_long_out(int ncol, int istr0, int N, const c_t<T>* __restrict__ z, const c_t<T>* __restrict__ twN,
                    const double* __restrict__ ginv, const float* __restrict__ ginvf, double* __restrict__ out,
                    float2* __restrict__ outff, int accumulate, const Ctl* __restrict__ ctl, double* __restrict__ dpart) {
    using C = c_t<T>;
    constexpr int CW = TimeCfg<T, NL>::CW, NTH = TimeCfg<T, NL>::NTH;
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* tw = buf + NL * CW;
    const int tid = threadIdx.x;
    const int o = blockIdx.y;
    const int j0 = blockIdx.x * CW;
    const int step = N / NL;
    const int nspace = 2 * ncol;
    for (int i = tid; i < NL; i += NTH) tw[i] = twN[(size_t)i * step];
    for (int e = tid; e < NL * CW; e += NTH) {
        const int c = e % CW, m = e / CW;
        buf[e] = j0 + c < ncol ? z[((size_t)m * istr0 + o) * ncol + j0 + c] : mkc(T(0), T(0));
    }
    __syncthreads();
    smem_fft<C, NL, +1, NTH, CW, CW, 1>(buf, tw);
    float d2 = 0.f, u2 = 0.f;
    const bool want = dpart != nullptr;
    for (int e = tid; e < NL * CW; e += NTH) {
        const int c = e % CW, m = e / CW;
        const int j = j0 + c;
        if (j >= ncol) continue;
        const size_t n = (size_t)m * istr0 + o;
        const C v = buf[e];
        if constexpr (OUTK == 1) {
            const float gi = ginvf[n];
            float2* row = outff + n * nspace;
            const float da = (float)v.x * gi, db = (float)v.y * gi;
            const float2 wa = ff_add_f(row[2 * j], da), wb = ff_add_f(row[2 * j + 1], db);
            row[2 * j] = wa;
            row[2 * j + 1] = wb;
            if (want) {
                d2 = fmaf(da, da, fmaf(db, db, d2));
                u2 = fmaf(wa.x, wa.x, fmaf(wb.x, wb.x, u2));
            }
        } else {
            const double gi = ginv[n];
            double* row = out + n * nspace;
            const double da = (double)v.x * gi, db = (double)v.y * gi;
            if (accumulate) {
                const double wa = row[2 * j] + da, wb = row[2 * j + 1] + db;
                row[2 * j] = wa;
                row[2 * j + 1] = wb;
                if (want) {
                    d2 = fmaf((float)da, (float)da, fmaf((float)db, (float)db, d2));
                    u2 = fmaf((float)wa, (float)wa, fmaf((float)wb, (float)wb, u2));
                }
            } else {
                row[2 * j] = da;
                row[2 * j + 1] = db;
            }
        }
    }
    if (want) {
        __shared__ double red[2][32];
        double a = warp_sum((double)d2), b = warp_sum((double)u2);
        if (tid % 32 == 0) { red[0][tid / 32] = a; red[1][tid / 32] = b; }
        __syncthreads();
        if (tid == 0) {
            double A = 0.0, B = 0.0;
            for (int w = 0; w < NTH / 32; ++w) { A += red[0][w]; B += red[1][w]; }
            const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
            dpart[2 * cta] = A;
            dpart[2 * cta + 1] = B;
        }
    }
}

template <class T, int NT>
static cudaError_t configure_time() {
    const int sm = (int)TimeCfg<T, NT>::SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_time_fwd<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_time_inv<T, NT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) {
        e = cudaFuncSetAttribute(k_time_inv<T, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        if constexpr (NT <= 512)
            e = cudaFuncSetAttribute(k_time_inv_ff_tma<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TimeTmaCfg<NT>::SMEM);
    }
    return e;
}

template <class T, int NL>
static cudaError_t configure_long() {
    const int sm = (int)TimeCfg<T, NL>::SMEM;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_time_long_pass<T, NL, -1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_time_long_pass<T, NL, -1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_time_long_pass<T, NL, +1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_time_long_out<T, NL, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if constexpr (sizeof(T) == 4)
        if ((e = cudaFuncSetAttribute(k_time_long_out<T, NL, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
            return e;
    return cudaSuccess;
}

template <class T>
cudaError_t configure_time_all() {
    cudaError_t e;
    if ((e = configure_long<T, 32>()) || (e = configure_long<T, 64>()) || (e = configure_long<T, 128>()) ||
        (e = configure_long<T, 256>()))
        return e;
#define PINT_CFG(NT) if ((e = configure_time<T, NT>()) != cudaSuccess) return e;
    PINT_CFG(2) PINT_CFG(4) PINT_CFG(8) PINT_CFG(16) PINT_CFG(32) PINT_CFG(64) PINT_CFG(128) PINT_CFG(256)
    PINT_CFG(512) PINT_CFG(1024)
#undef PINT_CFG
    return cudaSuccess;
}
template cudaError_t configure_time_all<float>();
template cudaError_t configure_time_all<double>();

template <class T, int NT>
static void time_fwd_nt(int nspace, const T* s, c_t<T>* S, const c_t<T>* twt, const Ctl* ctl, cudaStream_t st) {
    constexpr int CW = TimeCfg<T, NT>::CW;
    int grid = (nspace + 2 * CW - 1) / (2 * CW);
    launch_pdl(k_time_fwd<T, NT>, dim3(grid), dim3(TimeCfg<T, NT>::NTH), TimeCfg<T, NT>::SMEM, st, nspace, s, S, twt, ctl);
}
template <class T, int NT>
static void time_inv_nt(int nspace, const c_t<T>* S, const c_t<T>* twt, const double* ginv, double* out, int acc,
                        const Ctl* ctl, double* dpart, cudaStream_t st) {
    constexpr int CW = TimeCfg<T, NT>::CW;
    int grid = (nspace + 2 * CW - 1) / (2 * CW);
    k_time_inv<T, NT, 0><<<grid, TimeCfg<T, NT>::NTH, TimeCfg<T, NT>::SMEM, st>>>(nspace, S, twt, ginv, nullptr, out,
                                                                                  nullptr, acc, ctl, dpart);
}
// The prefetching kernel serves even point counts and N_t <= 512 (it needs a control block for its status).
static bool time_inv_ff_prefetch(int nt, int nspace, const Ctl* ctl) {
    return ctl != nullptr && nspace % 2 == 0 && nt <= 512;
}

template <int NT>
static void time_inv_ff_nt(int nspace, const float2* S, const float2* twt, const float* ginvf, float2* Uff,
                           const Ctl* ctl, double* dpart, cudaStream_t st) {
    if constexpr (NT <= 512) {
        if (time_inv_ff_prefetch(NT, nspace, ctl)) {
            using Cfg = TimeTmaCfg<NT>;
            const int grid = (nspace + 2 * Cfg::CW - 1) / (2 * Cfg::CW);
            launch_pdl(k_time_inv_ff_tma<NT>, dim3(grid), dim3(Cfg::NTH), Cfg::SMEM, st, nspace, S, twt, ginvf, Uff, ctl,
                       dpart);
            return;
        }
    }
    constexpr int CW = TimeCfg<float, NT>::CW;
    int grid = (nspace + 2 * CW - 1) / (2 * CW);
    k_time_inv<float, NT, 1><<<grid, TimeCfg<float, NT>::NTH, TimeCfg<float, NT>::SMEM, st>>>(
        nspace, S, twt, nullptr, ginvf, nullptr, Uff, 1, ctl, dpart);
}

// ---- long time axes: host side ----
// Forward pass s (kind 0: with twiddle, 1: the last, without) or inverse pass
// s >= 1 (kind 2: with the twiddle of pass s-1).
template <class T, int NL>
static void long_pass_nl(int kind, int ncol, int istr, int fprev, int N, c_t<T>* z, const c_t<T>* twN,
                         const Ctl* ctl, cudaStream_t st) {
    using Cfg = TimeCfg<T, NL>;
    dim3 grid((ncol + Cfg::CW - 1) / Cfg::CW, N / NL);
    if (kind == 0) k_time_long_pass<T, NL, -1, true><<<grid, Cfg::NTH, Cfg::SMEM, st>>>(ncol, istr, 1, N, z, twN, ctl);
    else if (kind == 1) k_time_long_pass<T, NL, -1, false><<<grid, Cfg::NTH, Cfg::SMEM, st>>>(ncol, istr, 1, N, z, twN, ctl);
    else k_time_long_pass<T, NL, +1, true><<<grid, Cfg::NTH, Cfg::SMEM, st>>>(ncol, istr, fprev, N, z, twN, ctl);
}
template <class T>
static cudaError_t long_pass(int kind, int nl, int ncol, int istr, int fprev, int N, c_t<T>* z, const c_t<T>* twN,
                             const Ctl* ctl, cudaStream_t st) {
    switch (nl) {
        case 32: long_pass_nl<T, 32>(kind, ncol, istr, fprev, N, z, twN, ctl, st); break;
        case 64: long_pass_nl<T, 64>(kind, ncol, istr, fprev, N, z, twN, ctl, st); break;
        case 128: long_pass_nl<T, 128>(kind, ncol, istr, fprev, N, z, twN, ctl, st); break;
        case 256: long_pass_nl<T, 256>(kind, ncol, istr, fprev, N, z, twN, ctl, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}
// CTAs of the unpack / pack kernels for `rows` rows of ncol columns (grid-stride beyond 8 waves).
static int pack_grid(int rows, int ncol) {
    const int rb = ncol <= kPackThreads ? kPackThreads / ncol : 1;
    const long b = (rows + rb - 1) / rb;
    return (int)(b > 8L * 152 * 8 ? 8L * 152 * 8 : (b < 1 ? 1 : b));
}

template <class T>
static cudaError_t time_fwd_long(int nt, int nspace, T* s, c_t<T>* S, const c_t<T>* twt, const Ctl* ctl,
                                 cudaStream_t st) {
    const LongPlan pl = long_plan(nt);
    const int ncol = nspace / 2;
    c_t<T>* z = reinterpret_cast<c_t<T>*>(s);   // s is consumed here: the workspace is s itself
    cudaError_t e;
    for (int i = 0; i < pl.S; ++i)
        if ((e = long_pass<T>(i + 1 < pl.S ? 0 : 1, pl.f[i], ncol, pl.istr[i], 1, nt, z, twt, ctl, st))) return e;
    k_time_long_unpack<T><<<pack_grid(nt / 2 + 1, ncol), kPackThreads, 0, st>>>(nt, pl, ncol, z, S, ctl);
    return cudaGetLastError();
}

template <class T, int NL, int OUTK>
static void long_out_nl(int ncol, int istr0, int N, const c_t<T>* z, const c_t<T>* twN, const double* ginv,
                        const float* ginvf, double* out, float2* outff, int acc, const Ctl* ctl, double* dpart,
                        cudaStream_t st) {
    using Cfg = TimeCfg<T, NL>;
    dim3 grid((ncol + Cfg::CW - 1) / Cfg::CW, istr0);
    k_time_long_out<T, NL, OUTK><<<grid, Cfg::NTH, Cfg::SMEM, st>>>(ncol, istr0, N, z, twN, ginv, ginvf, out, outff,
                                                                   acc, ctl, dpart);
}
template <class T, int OUTK>
static cudaError_t time_inv_long(int nt, int nspace, const c_t<T>* S, const c_t<T>* twt, void* work,
                                 const double* ginv, const float* ginvf, double* out, float2* outff, int acc,
                                 const Ctl* ctl, double* dpart, cudaStream_t st, const LongSolve<T>* ls) {
    if (!work) return cudaErrorInvalidValue;
    const LongPlan pl = long_plan(nt);
    const int ncol = nspace / 2;
    c_t<T>* z = reinterpret_cast<c_t<T>*>(work);
    cudaError_t e;
    if (ls) {
        if ((e = launch_long_pack_solve<T>(nt, S, z, *ls, ctl, st))) return e;
    } else {
        k_time_long_pack<T><<<pack_grid(nt, ncol), kPackThreads, 0, st>>>(nt, pl, ncol, S, z, ctl);
    }
    for (int i = pl.S - 1; i >= 1; --i)
        if ((e = long_pass<T>(2, pl.f[i], ncol, pl.istr[i], pl.f[i - 1], nt, z, twt, ctl, st))) return e;
    const int istr0 = pl.istr[0];
    switch (pl.f[0]) {
        case 32: long_out_nl<T, 32, OUTK>(ncol, istr0, nt, z, twt, ginv, ginvf, out, outff, acc, ctl, dpart, st); break;
        case 64: long_out_nl<T, 64, OUTK>(ncol, istr0, nt, z, twt, ginv, ginvf, out, outff, acc, ctl, dpart, st); break;
        case 128: long_out_nl<T, 128, OUTK>(ncol, istr0, nt, z, twt, ginv, ginvf, out, outff, acc, ctl, dpart, st); break;
        case 256: long_out_nl<T, 256, OUTK>(ncol, istr0, nt, z, twt, ginv, ginvf, out, outff, acc, ctl, dpart, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// CTAs (dpart pairs) of the output pass of a long time axis.
static int time_long_blocks(int nt, int nspace, int f32) {
    const LongPlan pl = long_plan(nt);
    int cw = 32;
    switch (pl.f[0]) {
#define CW_(N) case N: cw = f32 ? TimeCfg<float, N>::CW : TimeCfg<double, N>::CW; break;
        CW_(32) CW_(64) CW_(128) CW_(256)
#undef CW_
        default: break;
    }
    return (nspace / 2 + cw - 1) / cw * pl.istr[0];
}

// passes + unpack; pack (or pack with the fused spatial solve) + passes 1.. + output pass
int time_fwd_launches(int nt) { return nt > 1024 ? long_plan(nt).S + 1 : 1; }
int time_inv_launches(int nt) { return nt > 1024 ? long_plan(nt).S + 1 : 1; }

int time_inv_ff_blocks(int nt, int nspace, const Ctl* ctl) {
    if (nt > 1024) return time_long_blocks(nt, nspace, 1);
    if (time_inv_ff_prefetch(nt, nspace, ctl)) return (nspace + 31) / 32;
    return time_inv_blocks(nt, nspace, 1);
}

int time_inv_blocks(int nt, int nspace, int f32) {
    if (nt > 1024) return time_long_blocks(nt, nspace, f32);
    int cw = 32;
    switch (nt) {
#define CW_(N) case N: cw = f32 ? TimeCfg<float, N>::CW : TimeCfg<double, N>::CW; break;
        CW_(2) CW_(4) CW_(8) CW_(16) CW_(32) CW_(64) CW_(128) CW_(256) CW_(512) CW_(1024)
#undef CW_
        default: break;
    }
    return (nspace + 2 * cw - 1) / (2 * cw);
}

#define PINT_NT_SWITCH(CALL)                                                                            \
    switch (nt) {                                                                                       \
        case 2: CALL(2); break;     case 4: CALL(4); break;     case 8: CALL(8); break;                 \
        case 16: CALL(16); break;   case 32: CALL(32); break;   case 64: CALL(64); break;               \
        case 128: CALL(128); break; case 256: CALL(256); break; case 512: CALL(512); break;             \
        case 1024: CALL(1024); break;                                                                   \
        default: return cudaErrorInvalidValue;                                                          \
    }

template <class T>
cudaError_t launch_time_fwd(int nt, int nspace, const T* s, c_t<T>* S, const c_t<T>* twt, const Ctl* ctl,
                            cudaStream_t st) {
    if (nt > 1024) return time_fwd_long<T>(nt, nspace, const_cast<T*>(s), S, twt, ctl, st);
#define CALL(N) time_fwd_nt<T, N>(nspace, s, S, twt, ctl, st)
    PINT_NT_SWITCH(CALL)
#undef CALL
    return cudaGetLastError();
}
template <class T>
cudaError_t launch_time_inv(int nt, int nspace, const c_t<T>* S, const c_t<T>* twt, const double* ginv, double* out,
                            int accumulate, const Ctl* ctl, double* dpart, cudaStream_t st, void* work,
                            const LongSolve<T>* ls) {
    if (nt > 1024)
        return time_inv_long<T, 0>(nt, nspace, S, twt, work, ginv, nullptr, out, nullptr, accumulate, ctl, dpart, st,
                                   ls);
    if (ls) return cudaErrorInvalidValue;
#define CALL(N) time_inv_nt<T, N>(nspace, S, twt, ginv, out, accumulate, ctl, dpart, st)
    PINT_NT_SWITCH(CALL)
#undef CALL
    return cudaGetLastError();
}

cudaError_t launch_time_inv_ff(int nt, int nspace, const float2* S, const float2* twt, const float* ginvf,
                               float2* Uff, const Ctl* ctl, double* dpart, cudaStream_t st, void* work,
                               const LongSolve<float>* ls) {
    if (nt > 1024)
        return time_inv_long<float, 1>(nt, nspace, S, twt, work, nullptr, ginvf, nullptr, Uff, 1, ctl, dpart, st, ls);
    if (ls) return cudaErrorInvalidValue;
#define CALL(N) time_inv_ff_nt<N>(nspace, S, twt, ginvf, Uff, ctl, dpart, st)
    PINT_NT_SWITCH(CALL)
#undef CALL
    return cudaGetLastError();
}

template cudaError_t launch_time_fwd<float>(int, int, const float*, float2*, const float2*, const Ctl*, cudaStream_t);
template cudaError_t launch_time_fwd<double>(int, int, const double*, double2*, const double2*, const Ctl*,
                                             cudaStream_t);
template cudaError_t launch_time_inv<float>(int, int, const float2*, const float2*, const double*, double*, int,
                                            const Ctl*, double*, cudaStream_t, void*, const LongSolve<float>*);
template cudaError_t launch_time_inv<double>(int, int, const double2*, const double2*, const double*, double*, int,
                                             const Ctl*, double*, cudaStream_t, void*, const LongSolve<double>*);

}  // namespace pint
