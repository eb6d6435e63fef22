// k_timegemm.cu - Steps 1 and 3 of the diagonalized solve (Eq. 2.8) as dense
// DFT matrix products on the tensor cores (tcgen05, accumulators in TMEM), for
// time axes of N_t = 64 or 128 steps.
//
// Forward (Step 1):  S_k[p] = sum_n s_n[p] e^{-2 pi i n k / N_t},  k = 0..N_t/2
// (s already alpha-scaled), is D = A W^T with A[p][n] = s_n[p] (one row per
// spatial point) and W the real DFT matrix of N_t rows: the cosine rows of
// k = 0..N_t/2 and the negated sine rows of k = 1..N_t/2-1, interleaved as
// (cos_0, cos_{N/2}, cos_1, -sin_1, cos_2, -sin_2, ...), so that each output
// pair of columns is one complex S_k.
// Inverse (Step 3):  x_n[p] = sum_k c_k (Re S_k cos(2 pi n k/N) - Im S_k sin(2 pi n k/N))
// (c_0 = c_{N/2} = 1, else 2: the Hermitian half spectrum), then
// U_n += gamma_n^{-1} x_n / N_t in one FP64 fused multiply-add (the unscaling
// and the update of Step 3).  The input row of point p holds (Re S_0, Re S_{N/2},
// Re S_1, Im S_1, ...), i.e. the half spectrum in its stored complex order.
//
// Precision (split FP16, FP32 accumulation): each point's row is scaled by a
// power of two so that its largest entry lies in [2^13, 2^14), split into
// hi = fp16(x), lo = fp16(x - hi), and so is W; D = A_hi W_hi + A_hi W_lo +
// A_lo W_hi.  Every entry is then represented to about 2^-22 of its row's
// largest one (FP16 subnormals keep the absolute spacing 2^-24 of the scaled
// row), the accuracy of the FP32 FFT it stands in for; the scale is undone on
// the FP32 result.
//
// Tiles: 128 spatial points (the MMA's M, one TMEM lane per point) x all N_t
// levels.  One CTA per SM walks its tiles: a bulk asynchronous copy brings the
// next tile into the staging buffer while the current one is multiplied, and
// the epilogue of the previous tile (TMEM -> HBM) runs while the tensor cores
// work on the current one (two TMEM accumulators).  Operands live in shared
// memory in the K-major 128-byte-swizzled layout of the tcgen05 descriptors.
#include <cuda_fp16.h>

#include <vector>

#include "../../include/pint.h"
#include "pint_common.cuh"
#include "pint_kernels.h"
#include "tma.cuh"

namespace pint {

// Byte offset of element (row r, column k) of a K-major, 128-byte-swizzled
// tile of R rows of 16-bit elements: column blocks of 64 elements, each R x 128
// bytes; inside a block, groups of 8 rows of 1024 bytes, and the 16-byte chunk
// c of row r stored at chunk c ^ (r mod 8).
__host__ __device__ __forceinline__ uint32_t sw128_off(int r, int k, int R) {
    const int kb = k >> 6, byte = (k & 63) * 2;
    return (uint32_t)(kb * (R * 128) + (r >> 3) * 1024 + (r & 7) * 128 + ((((byte >> 4) ^ (r & 7))) << 4) + (byte & 15));
}

// Shared-memory matrix descriptor (tcgen05): start address, leading / stride
// byte offsets (16-byte units), version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused by this layout): 16 B
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
    d |= 1ull << 46;                           // descriptor version
    d |= 2ull << 61;                           // 128-byte swizzle
    return d;
}
// Instruction descriptor: FP32 accumulator, FP16 A and B, both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 consecutive TMEM columns of this warp's 32 lanes (lane = thread), one FP32 each.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 2^e as a float for e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
// Exponent e with 2^(e-1) <= |x| < 2^e for the largest |x| given its float bits (0 for zero).
__device__ __forceinline__ int fexp_bits(uint32_t absbits) { return (int)(absbits >> 23) - 126; }

template <int NT, bool INV> struct GemmCfg {
    static constexpr int M = 128;                                // points per tile
    static constexpr int KDIM = NT;                              // reduction length
    static constexpr int NCOL = NT;                              // output columns
    static constexpr int NTH = 256;
    static constexpr size_t B_BYTES = (size_t)NCOL * KDIM * 2;   // one split of W
    static constexpr size_t A_BYTES = (size_t)M * KDIM * 2;
    static constexpr int SROWS = INV ? NT / 2 + 1 : NT;          // staging rows (levels or frequencies)
    static constexpr int SELEM = INV ? 8 : 4;                    // staging element bytes
    static constexpr size_t S_BYTES = (size_t)SROWS * M * SELEM;
    static constexpr size_t OFF_BH = 0, OFF_BL = B_BYTES, OFF_AH = 2 * B_BYTES, OFF_AL = 2 * B_BYTES + A_BYTES;
    static constexpr size_t OFF_ST = 2 * B_BYTES + 2 * A_BYTES;
    static constexpr size_t OFF_MISC = OFF_ST + S_BYTES;         // escale[2][128], pmax[2][128], barriers, tmem
    static constexpr size_t SMEM = OFF_MISC + 2 * 128 * 4 + 2 * 128 * 4 + 64 + 1024;   // + alignment slack
    static constexpr uint32_t TMEM_COLS = 2 * NCOL;              // two accumulators
};

// W in the forward interleaved order (row j of the N_t x N_t matrix acting on the time signal):
// j = 0: cos_0, j = 1: cos_{N/2}, j = 2k: cos_k, j = 2k+1: -sin_k (k >= 1).
// Inverse (row n of the matrix acting on the stored half spectrum, column j):
// j = 0: Re S_0 (c 1), j = 1: Re S_{N/2} (c 1), j = 2k: 2 cos, j = 2k+1: -2 sin.

template <int NT, bool INV>
__global__ void __launch_bounds__(256, 1)
    k_time_gemm(int nspace, int ntiles, const void* __restrict__ src, void* __restrict__ dst,
                const __half* __restrict__ w_hi, const __half* __restrict__ w_lo, const double* __restrict__ ginv,
                Ctl* __restrict__ ctl, double* __restrict__ dpart) {
    using Cfg = GemmCfg<NT, INV>;
    constexpr int M = Cfg::M, KD = Cfg::KDIM, NC = Cfg::NCOL, NTH = Cfg::NTH, SROWS = Cfg::SROWS;
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sBh = sm + Cfg::OFF_BH;
    unsigned char* sBl = sm + Cfg::OFF_BL;
    unsigned char* sAh = sm + Cfg::OFF_AH;
    unsigned char* sAl = sm + Cfg::OFF_AL;
    unsigned char* stg = sm + Cfg::OFF_ST;
    int* escale = reinterpret_cast<int*>(sm + Cfg::OFF_MISC);               // [2][128]
    uint32_t* pmax = reinterpret_cast<uint32_t*>(escale + 256);            // [2][128]
    uint64_t* bar_ld = reinterpret_cast<uint64_t*>(pmax + 256);
    uint64_t* bar_mma = bar_ld + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_mma + 1);
    int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;

    // W (both splits) into the swizzled layout, once per CTA
    for (int i = tid; i < NC * KD / 8; i += NTH) {
        const int r = (i * 8) / KD, k = (i * 8) % KD;
        const uint4 h = *reinterpret_cast<const uint4*>(w_hi + (size_t)r * KD + k);
        const uint4 l = *reinterpret_cast<const uint4*>(w_lo + (size_t)r * KD + k);
        *reinterpret_cast<uint4*>(sBh + sw128_off(r, k, NC)) = h;
        *reinterpret_cast<uint4*>(sBl + sw128_off(r, k, NC)) = l;
    }
    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_mma, 1);
        mbar_fence_init();
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(Cfg::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_proxy_async_smem();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // issue the bulk copies of tile t into the staging buffer (warp 0)
    auto issue_load = [&](int t) {
        const long p0 = (long)t * M;
        const int npts = (int)min((long)M, (long)nspace - p0);
        const uint32_t rowb = (uint32_t)npts * Cfg::SELEM;
        if (lane == 0) mbar_arrive_expect_tx(bar_ld, rowb * SROWS);
        __syncwarp();
        for (int r = lane; r < SROWS; r += 32) {
            const unsigned char* g = reinterpret_cast<const unsigned char*>(src) + ((size_t)r * nspace + p0) * Cfg::SELEM;
            bulk_g2s(stg + (size_t)r * M * Cfg::SELEM, g, rowb, bar_ld);
        }
    };

    int ti = 0;                  // local tile counter
    int t = blockIdx.x;
    if (t < ntiles && warp == 0) issue_load(t);
    float d2 = 0.f, u2 = 0.f;    // update-size partials (inverse, when dpart != nullptr)
    const bool want = INV && dpart != nullptr;
    bool ok = true;
    // epilogue of local tile e (global tile tg), accumulator buffer e & 1
    auto epilogue = [&](int e, int tg) {
        const int q = 32 * (warp & 3) + lane;            // point (TMEM lane) of this thread
        const int ch = warp >> 2;                        // column half
        const long p = (long)tg * M + q;
        const bool in = p < nspace;
        const uint32_t base = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((e & 1) * NC + ch * (NC / 2));
        const float sc = pow2f(escale[(e & 1) * 128 + q]);
#pragma unroll 1
        for (int c0 = 0; c0 < NC / 2; c0 += 32) {
            const int cb = ch * (NC / 2) + c0;            // first output column of this chunk
            if constexpr (!INV) {
                float v[32];
                tmem_ld32(base + c0, v);
                if (in) {
                    float2* S = reinterpret_cast<float2*>(dst);
                    if (cb == 0) {                        // columns 0, 1: S_0 and S_{N/2} (real)
                        S[p] = make_float2(v[0] * sc, 0.f);
                        S[(size_t)(NT / 2) * nspace + p] = make_float2(v[1] * sc, 0.f);
                    } else {
                        S[(size_t)(cb >> 1) * nspace + p] = make_float2(v[0] * sc, v[1] * sc);
                    }
#pragma unroll
                    for (int i = 2; i < 32; i += 2)
                        S[(size_t)((cb + i) >> 1) * nspace + p] = make_float2(v[i] * sc, v[i + 1] * sc);
                }
            } else {
                // the iterate's 32 levels first (independent loads in flight), then the accumulators
                double* U = reinterpret_cast<double*>(dst);
                double uo[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) uo[i] = in ? __ldcs(U + (size_t)(cb + i) * nspace + p) : 0.0;
                float v[32];
                tmem_ld32(base + c0, v);
                if (in) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int n = cb + i;
                        const double w = fma(f32_to_f64_exact(v[i] * sc), ginv[n], uo[i]);
                        __stcs(U + (size_t)n * nspace + p, w);
                        if (want) {
                            const float dl = v[i] * sc * f64_to_f32_trunc(ginv[n]), wf = f64_to_f32_trunc(w);
                            d2 = fmaf(dl, dl, d2);
                            u2 = fmaf(wf, wf, u2);
                        }
                    }
                }
            }
        }
    };

    int prev_tile = -1;
    for (; t < ntiles && ok; t += gridDim.x, ++ti) {
        // staging of tile t has landed; the accumulator of tile t-2 and operand A are free
        ok = __syncthreads_and(mbar_wait_bounded(bar_ld, ti & 1));
        if (!ok) break;
        if (ti > 0) {
            ok = __syncthreads_and(mbar_wait_bounded(bar_mma, (ti - 1) & 1));   // MMA of the previous tile done
            if (!ok) break;
        }
        // ---- convert: per-point scale, split into FP16 hi / lo, K-major swizzled A ----
        {
            const int q = tid & 127, h = tid >> 7;       // point, half of the row
            uint32_t mx = 0;
            if constexpr (!INV) {
                const float* st = reinterpret_cast<const float*>(stg);
                for (int n = h * (KD / 2); n < (h + 1) * (KD / 2); ++n) mx = max(mx, __float_as_uint(st[n * M + q]) & 0x7FFFFFFFu);
            } else {
                const float2* st = reinterpret_cast<const float2*>(stg);
                for (int k = h * (NT / 4); k < (h + 1) * (NT / 4) + (h ? 1 : 0); ++k) {
                    const float2 z = st[k * M + q];
                    mx = max(mx, __float_as_uint(z.x) & 0x7FFFFFFFu);
                    if (k > 0 && k < NT / 2) mx = max(mx, __float_as_uint(z.y) & 0x7FFFFFFFu);
                }
            }
            pmax[h * 128 + q] = mx;
            __syncthreads();
            const uint32_t m2 = max(pmax[q], pmax[128 + q]);
            const int e = m2 == 0u ? 0 : min(max(fexp_bits(m2), -100), 100);
            const float up = pow2f(14 - e);              // the row's largest entry into [2^13, 2^14)
            if (h == 0) escale[(ti & 1) * 128 + q] = e - 14;
            for (int kc = h * (KD / 2); kc < (h + 1) * (KD / 2); kc += 8) {
                float x[8];
                if constexpr (!INV) {
                    const float* st = reinterpret_cast<const float*>(stg);
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = st[(kc + i) * M + q];
                } else {
                    // columns kc .. kc+7 = (Re, Im) of frequencies kc/2 .. kc/2+3; column 1 holds Re S_{N/2}
                    const float2* st = reinterpret_cast<const float2*>(stg);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k = kc / 2 + i;
                        const float2 z = st[k * M + q];
                        x[2 * i] = z.x;
                        x[2 * i + 1] = z.y;
                    }
                    if (kc == 0) x[1] = st[(NT / 2) * M + q].x;
                }
                __half hv[8], lv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float y = x[i] * up;
                    hv[i] = __float2half_rn(y);
                    lv[i] = __float2half_rn(y - __half2float(hv[i]));
                }
                *reinterpret_cast<uint4*>(sAh + sw128_off(q, kc, M)) = *reinterpret_cast<const uint4*>(hv);
                *reinterpret_cast<uint4*>(sAl + sw128_off(q, kc, M)) = *reinterpret_cast<const uint4*>(lv);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();                                  // A written; staging consumed
        // ---- next tile's copies, then this tile's MMAs ----
        if (warp == 0 && t + (int)gridDim.x < ntiles) issue_load(t + gridDim.x);
        if (tid == 0) {
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)((ti & 1) * NC);
            constexpr uint32_t idesc = umma_idesc_f16(NC);
            const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {             // A_hi W_hi, A_hi W_lo, A_lo W_hi
                const uint32_t a = pr < 2 ? ah : al, b = pr == 1 ? bl : bh;
#pragma unroll
                for (int s = 0; s < KD / 16; ++s) {
                    const uint32_t oa = (uint32_t)((s >> 2) * (M * 128) + (s & 3) * 32);
                    const uint32_t ob = (uint32_t)((s >> 2) * (NC * 128) + (s & 3) * 32);
                    umma_f16(d, umma_sdesc(a + oa), umma_sdesc(b + ob), idesc, (pr | s) ? 1u : 0u);
                }
            }
            umma_commit(bar_mma);
        }
        // ---- epilogue of the previous tile, overlapping this tile's MMAs and the next copies ----
        if (prev_tile >= 0) {
            epilogue(ti - 1, prev_tile);
            tc_fence_before();
        }
        prev_tile = t;
    }
    if (ok && prev_tile >= 0) {
        ok = __syncthreads_and(mbar_wait_bounded(bar_mma, (ti - 1) & 1));
        if (ok) {
            tc_fence_after();
            epilogue(ti - 1, prev_tile);
            tc_fence_before();
        }
    }
    if (!ok && tid == 0) {
        if (ctl) atomicExch(&ctl->status, (int)PINT_ECUDA);
        *abort_flag = 1;
    }
    __syncthreads();
    if (*abort_flag) {
        // let whatever is in flight land before the CTA's memory goes away
        if (tid == 0) {
            mbar_wait_bounded(bar_ld, ti & 1);
            mbar_wait_bounded(bar_mma, (ti - 1) & 1);
        }
        __syncthreads();
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS));
    if (want) {
        __shared__ double red[2][8];
        double a = warp_sum((double)d2), b = warp_sum((double)u2);
        if (lane == 0) { red[0][warp] = a; red[1][warp] = b; }
        __syncthreads();
        if (tid == 0) {
            double A = 0.0, B = 0.0;
            for (int w = 0; w < 8; ++w) { A += red[0][w]; B += red[1][w]; }
            dpart[2 * blockIdx.x] = A;
            dpart[2 * blockIdx.x + 1] = B;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int time_gemm_supported(int nt, int nspace) { return (nt == 64 || nt == 128) && nspace % 4 == 0; }

int time_gemm_blocks(int nspace) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (nspace + 127) / 128;
    return ntiles < sms ? ntiles : sms;
}

// W tables (FP16 hi and lo parts, row-major [row][column]) of both directions for one N_t:
// forward first (nt x nt), then inverse (nt x nt), each as hi then lo.
void time_gemm_tables(int nt, std::vector<uint16_t>& out) {
    out.assign((size_t)4 * nt * nt, 0);
    auto put = [&](size_t off, int r, int c, double w) {
        const __half h = __double2half(w);
        const __half l = __double2half(w - (double)__half2float(h));
        out[off + (size_t)r * nt + c] = *reinterpret_cast<const uint16_t*>(&h);
        out[off + (size_t)nt * nt + (size_t)r * nt + c] = *reinterpret_cast<const uint16_t*>(&l);
    };
    const double tau = 2.0 * M_PI / nt;
    for (int j = 0; j < nt; ++j) {
        for (int n = 0; n < nt; ++n) {
            // forward row j acting on level n
            double wf;
            if (j == 0) wf = 1.0;
            else if (j == 1) wf = (n % 2 == 0) ? 1.0 : -1.0;                    // cos(pi n)
            else if (j % 2 == 0) wf = cos(tau * ((long)n * (j / 2) % nt));
            else wf = -sin(tau * ((long)n * (j / 2) % nt));
            put(0, j, n, wf);
            // inverse row n acting on spectrum column j
            double wi;
            if (j == 0) wi = 1.0;
            else if (j == 1) wi = (n % 2 == 0) ? 1.0 : -1.0;
            else if (j % 2 == 0) wi = 2.0 * cos(tau * ((long)n * (j / 2) % nt));
            else wi = -2.0 * sin(tau * ((long)n * (j / 2) % nt));
            put((size_t)2 * nt * nt, n, j, wi);
        }
    }
}

template <int NT, bool INV>
static cudaError_t launch_gemm_t(int nspace, const void* src, void* dst, const __half* w, const double* ginv,
                                 Ctl* ctl, double* dpart, cudaStream_t st) {
    using Cfg = GemmCfg<NT, INV>;
    const int ntiles = (nspace + 127) / 128;
    const int blocks = time_gemm_blocks(nspace);
    const __half* wh = w + (INV ? (size_t)2 * NT * NT : 0);
    const __half* wl = wh + (size_t)NT * NT;
    return launch_pdl(k_time_gemm<NT, INV>, dim3(blocks), dim3(Cfg::NTH), Cfg::SMEM, st, nspace, ntiles, src, dst,
                      wh, wl, ginv, ctl, dpart);
}

cudaError_t launch_time_gemm(int inv, int nt, int nspace, const void* src, void* dst, const void* wtab,
                             const double* ginv, Ctl* ctl, double* dpart, cudaStream_t st) {
    const __half* w = reinterpret_cast<const __half*>(wtab);
    switch (nt) {
        case 64: return inv ? launch_gemm_t<64, true>(nspace, src, dst, w, ginv, ctl, dpart, st)
                            : launch_gemm_t<64, false>(nspace, src, dst, w, ginv, ctl, dpart, st);
        case 128: return inv ? launch_gemm_t<128, true>(nspace, src, dst, w, ginv, ctl, dpart, st)
                             : launch_gemm_t<128, false>(nspace, src, dst, w, ginv, ctl, dpart, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t configure_time_gemm() {
    cudaError_t e;
#define PINT_CFG_GEMM(NT, INV)                                                                           \
    if ((e = cudaFuncSetAttribute(k_time_gemm<NT, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)GemmCfg<NT, INV>::SMEM)) != cudaSuccess)                          \
        return e;
    PINT_CFG_GEMM(64, false)
    PINT_CFG_GEMM(64, true)
    PINT_CFG_GEMM(128, false)
    PINT_CFG_GEMM(128, true)
#undef PINT_CFG_GEMM
    return cudaSuccess;
}

}  // namespace pint
