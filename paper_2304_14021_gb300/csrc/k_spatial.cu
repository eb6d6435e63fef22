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
//  * sine (simply supported, n + 1 a power of two): DST-I by one complex FFT
//    of length 2(n+1) of the odd extension (k_dst.cu);
//  * dense (any other n <= 1024, and the vertex-centred DCT-I): X = F x,
//    x = F^{-1} X with the basis matrices held in device tables.
// 1-D: one fused pass (transform, divide, inverse) per row.  2-D: x-forward
// over rows, fused y pass (transform, divide, inverse) over columns, x-inverse.
#include <cooperative_groups.h>

#include "../../include/pint.h"
#include "colr_map.cuh"
#include "pint_common.cuh"
#include "pint_kernels.h"
#include "spatial.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace pint {

// Destination of MODE_PACK (1-D rows on a long time axis): the solved row
// S2[k] goes straight into the workspace of the inverse time transform as
// z[long_pos(k)][j] = S2[k][2j] + i S2[k][2j+1] and, for 0 < k < N_t/2, its
// Hermitian partner z[long_pos(N_t - k)][j] = conj(S2[k][2j]) + i conj(S2[k][2j+1]).
template <class T> struct PackDst {
    c_t<T>* z;
    LongPlan pl;
    int nt;
};


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
// Rows (x axis), cosine path.  A tile is ROWS consecutive rows of length N
// (contiguous in memory); row index gr = k * ny + y.  Persistent CTAs walk the
// tiles with a stride of gridDim.x through a ring of STAGES shared-memory
// buffers: tile loads are bulk asynchronous copies issued STAGES tiles ahead,
// so they overlap the FFTs of the tiles before them.
// ---------------------------------------------------------------------------
template <class T, int N> struct RowCfg {
    static constexpr int ROWS = N >= 2048 ? 1 : 2048 / N;
    static constexpr int NTH = 256;
    static constexpr int STAGES = 2;
    static constexpr int TILE = ROWS * N;                                   // elements
    static constexpr size_t BAR_OFF = sizeof(c_t<T>) * (size_t)STAGES * TILE;
    static constexpr size_t SMEM = BAR_OFF + 8 * STAGES;
    // resident CTAs per SM the register allocation is sized for
    static constexpr int MINB = sizeof(T) == 4 ? (N >= 2048 ? 3 : 4) : 2;
};

// Records a failed (timed out) barrier wait in the control block.
__device__ __forceinline__ void note_timeout(const Ctl* ctl) {
    if (ctl) atomicExch(const_cast<int*>(&ctl->status), (int)PINT_ECUDA);
}

template <class T, int N, int MODE>
__global__ void __launch_bounds__(256, RowCfg<T, N>::MINB) k_rows_dct(int nrows, int ny, c_t<T>* __restrict__ S, Tabs<T> tb,
                                                  SolveCoef co, const Ctl* __restrict__ ctl, PackDst<T> pd) {
    using C = c_t<T>;
    using Cfg = RowCfg<T, N>;
    constexpr int ROWS = Cfg::ROWS, NTH = Cfg::NTH, STAGES = Cfg::STAGES, TILE = Cfg::TILE;
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* bufs = reinterpret_cast<C*>(smem_raw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + Cfg::BAR_OFF);
    const int tid = threadIdx.x;
    const int ntiles = (nrows + ROWS - 1) / ROWS;
    // thread 0: post the byte count of tile t on stage st's barrier and start its copy
    auto issue = [&](int t, int st) {
        const long r0 = (long)t * ROWS;
        const uint32_t bytes = (uint32_t)(min((long)ROWS, nrows - r0) * N * sizeof(C));
        mbar_arrive_expect_tx(&bar[st], bytes);
        bulk_g2s(bufs + st * TILE, S + r0 * N, bytes, &bar[st]);
    };
    if (tid == 0) {
        for (int st = 0; st < STAGES; ++st) mbar_init(&bar[st], 1);
        mbar_fence_init();
        for (int st = 0; st < STAGES; ++st)
            if (blockIdx.x + st * gridDim.x < ntiles) issue(blockIdx.x + st * gridDim.x, st);
    }
    __syncthreads();
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int st = it % STAGES;
        C* buf = bufs + st * TILE;
        const bool ok = mbar_wait_bounded(&bar[st], (uint32_t)(it / STAGES) & 1u);
        if (!__syncthreads_and(ok)) {
            // give up: record the failure, let the copies still in flight land, stop
            if (tid == 0) {
                note_timeout(ctl);
                for (int k = 0; k < STAGES; ++k)
                    if (t + k * gridDim.x < ntiles)
                        mbar_wait_bounded(&bar[(it + k) % STAGES], (uint32_t)((it + k) / STAGES) & 1u);
            }
            __syncthreads();
            return;
        }
        const long r0 = (long)t * ROWS;
        // The tile arrives in natural order; the FFTs keep it swizzled (swz<1>).
        if constexpr (MODE == MODE_INV) {
            // pre-twiddle X -> V, read in natural order, written back swizzled
            constexpr int NP = ROWS * (N / 2 + 1), PPT = (NP + NTH - 1) / NTH;
            C vp[PPT], vq[PPT];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int e = tid + k * NTH;
                if (e < NP) {
                    const int b = e / (N / 2 + 1), p = e % (N / 2 + 1), q = (N - p) % N;
                    const C* row = buf + b * N;
                    dct_pre(p, row[p], row[q], tb.wx[p], tb.wx[q], vp[k], vq[k]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int e = tid + k * NTH;
                if (e < NP) {
                    const int b = e / (N / 2 + 1), p = e % (N / 2 + 1), q = (N - p) % N;
                    C* row = buf + b * N;
                    row[swz<1>(p)] = vp[k];
                    row[swz<1>(q)] = vq[k];
                }
            }
            __syncthreads();
        } else {
            smem_fft<C, N, -1, NTH, ROWS, 1, N, 1, true>(buf, tb.twx);
            for (int e = tid; e < ROWS * (N / 2 + 1); e += NTH) {
                const int b = e / (N / 2 + 1), p = e % (N / 2 + 1), q = (N - p) % N;
                C* row = buf + b * N;
                const int sp = swz<1>(p), sq = swz<1>(q);
                const C wp = tb.wx[p], wq = tb.wx[q];
                C Xp, Xq;
                dct_post(row[sp], row[sq], wp, wq, Xp, Xq);
                if (MODE == MODE_FDI || MODE == MODE_PACK) {
                    const int k = (int)((r0 + b) / ny);
                    if (r0 + b < nrows) {
                        Xp = cdiv(Xp, shift_den(tb, k, tb.lamx[p], c2, c1));
                        Xq = cdiv(Xq, shift_den(tb, k, tb.lamx[q], c2, c1));
                    }
                    dct_pre(p, Xp, Xq, wp, wq, Xp, Xq);
                }
                row[sp] = Xp;
                row[sq] = Xq;
            }
            __syncthreads();
        }
        if (MODE == MODE_FWD) {
#pragma unroll 4
            for (int e = tid; e < ROWS * N; e += NTH) {
                const long gr = r0 + e / N;
                if (gr < nrows) S[r0 * N + e] = buf[(e / N) * N + swz<1>(e % N)];
            }
        } else {
            smem_fft<C, N, +1, NTH, ROWS, 1, N, 1>(buf, tb.twx);
            const T inv = T(1) / T(N);
            if constexpr (MODE == MODE_PACK) {
                constexpr int NC = N / 2;
                const int half = pd.nt / 2;
                for (int e = tid; e < ROWS * NC; e += NTH) {
                    const int b = e / NC, j = e % NC;
                    const long k = r0 + b;
                    if (k >= nrows) continue;
                    C a = scalec(buf[b * N + swz<1>(dct_pos(2 * j, N))], inv);
                    C c = scalec(buf[b * N + swz<1>(dct_pos(2 * j + 1, N))], inv);
                    if (k == 0 || k == half) { a.y = T(0); c.y = T(0); }   // real in exact arithmetic
                    pd.z[(size_t)long_pos((int)k, pd.pl) * NC + j] = mkc(a.x - c.y, a.y + c.x);
                    if (k > 0 && k < half)
                        pd.z[(size_t)long_pos(pd.nt - (int)k, pd.pl) * NC + j] = mkc(a.x + c.y, c.x - a.y);
                }
            } else {
#pragma unroll 4
                for (int e = tid; e < ROWS * N; e += NTH) {
                    const int b = e / N, i = e % N;
                    const long gr = r0 + b;
                    if (gr < nrows) S[r0 * N + e] = scalec(buf[b * N + swz<1>(dct_pos(i, N))], inv);
                }
            }
        }
        fence_proxy_async_smem();   // this thread's accesses to buf precede the refill
        __syncthreads();            // every thread is done with buf
        if (tid == 0 && t + STAGES * gridDim.x < ntiles) issue(t + STAGES * gridDim.x, st);
    }
}

// ---------------------------------------------------------------------------
// Rows, warp-per-row form (128 <= N <= 512): every warp streams its own rows
// (row r = global warp id + i * all warps) through two shared-memory stages of
// its own, filled by bulk asynchronous copies one row ahead and completed on
// the warp's own mbarriers.  A warp synchronizes only with itself, so the
// warps of a CTA do not wait for one another at all.
// ---------------------------------------------------------------------------
template <class T, int N> struct RowWCfg {
    static constexpr int WARPS = 8, NTH = 32 * WARPS, STAGES = 2;
    static constexpr size_t ROWB = sizeof(c_t<T>) * N;
    static constexpr size_t BAR_OFF = (size_t)WARPS * STAGES * ROWB;
    static constexpr size_t SMEM = BAR_OFF + 8 * WARPS * STAGES;
    static constexpr int MINB = sizeof(T) == 4 && N <= 256 ? 4 : 2;
};
template <class T, int N>
constexpr bool rows_warp_ok = N >= 128 && N <= (sizeof(T) == 4 ? 512 : 256);

template <class T, int N, int MODE>
__global__ void __launch_bounds__(256, RowWCfg<T, N>::MINB) k_rows_dct_w(int nrows, int ny, c_t<T>* __restrict__ S,
                                                                         Tabs<T> tb, SolveCoef co,
                                                                         const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    using Cfg = RowWCfg<T, N>;
    constexpr int STAGES = Cfg::STAGES, NP = N / 2 + 1, PPL = (NP + 31) / 32;
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    C* mybuf = reinterpret_cast<C*>(smem_raw) + (size_t)warp * STAGES * N;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + Cfg::BAR_OFF) + warp * STAGES;
    const int gw = blockIdx.x * Cfg::WARPS + warp, nw = gridDim.x * Cfg::WARPS;
    auto issue = [&](int r, int st) {
        mbar_arrive_expect_tx(&bar[st], (uint32_t)Cfg::ROWB);
        bulk_g2s(mybuf + st * N, S + (size_t)r * N, (uint32_t)Cfg::ROWB, &bar[st]);
    };
    if (lane == 0) {
        for (int st = 0; st < STAGES; ++st) mbar_init(&bar[st], 1);
        mbar_fence_init();
        for (int st = 0; st < STAGES; ++st)
            if (gw + st * nw < nrows) issue(gw + st * nw, st);
    }
    __syncwarp();
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    int it = 0;
    for (int r = gw; r < nrows; r += nw, ++it) {
        const int st = it % STAGES;
        C* row = mybuf + st * N;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], (uint32_t)(it / STAGES) & 1u))) {
            if (lane == 0) {
                note_timeout(ctl);
                for (int k = 0; k < STAGES; ++k)
                    if (r + k * nw < nrows) mbar_wait_bounded(&bar[(it + k) % STAGES], (uint32_t)((it + k) / STAGES) & 1u);
            }
            __syncwarp();
            return;
        }
        if constexpr (MODE == MODE_INV) {
            // pre-twiddle X -> V, read in natural order, written back swizzled
            C vp[PPL], vq[PPL];
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const int p = lane + 32 * k, q = (N - p) % N;
                if (p < NP) dct_pre(p, row[p], row[q], tb.wx[p], tb.wx[q], vp[k], vq[k]);
            }
            __syncwarp();
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const int p = lane + 32 * k, q = (N - p) % N;
                if (p < NP) {
                    row[swz<1>(p)] = vp[k];
                    row[swz<1>(q)] = vq[k];
                }
            }
            __syncwarp();
        } else {
            warp_fft<C, N, -1, true, false>(row, tb.twx, lane);
            const int k = r / ny;
#pragma unroll
            for (int kk = 0; kk < PPL; ++kk) {
                const int p = lane + 32 * kk, q = (N - p) % N;
                if (p < NP) {
                    const int sp = swz<1>(p), sq = swz<1>(q);
                    const C wp = tb.wx[p], wq = tb.wx[q];
                    C Xp, Xq;
                    dct_post(row[sp], row[sq], wp, wq, Xp, Xq);
                    if (MODE == MODE_FDI) {
                        Xp = cdiv(Xp, shift_den(tb, k, tb.lamx[p], c2, c1));
                        Xq = cdiv(Xq, shift_den(tb, k, tb.lamx[q], c2, c1));
                        dct_pre(p, Xp, Xq, wp, wq, Xp, Xq);
                    }
                    row[sp] = Xp;
                    row[sq] = Xq;
                }
            }
            __syncwarp();
        }
        C* out = S + (size_t)r * N;
        if (MODE == MODE_FWD) {
#pragma unroll
            for (int i = lane; i < N; i += 32) out[i] = row[swz<1>(i)];
        } else {
            warp_fft<C, N, +1>(row, tb.twx, lane);
            const T inv = T(1) / T(N);
#pragma unroll
            for (int i = lane; i < N; i += 32) out[i] = scalec(row[swz<1>(dct_pos(i, N))], inv);
        }
        fence_proxy_async_smem();   // this lane's accesses to the stage precede the refill
        __syncwarp();
        if (lane == 0 && r + STAGES * nw < nrows) issue(r + STAGES * nw, st);
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
    static constexpr size_t TILE = sizeof(c_t<T>) * (size_t)N * CW;
    static constexpr int STAGES = 2 * TILE <= 160 * 1024 ? 2 : 1;
    static constexpr size_t SMEM = STAGES * TILE;
};

// cp.async of one complex value (8 or 16 bytes), global -> shared.
template <int BYTES>
__device__ __forceinline__ void cp_async_val(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit_grp() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N_PENDING> __device__ __forceinline__ void cp_async_wait_grp() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N_PENDING) : "memory");
}

// Persistent CTAs over tiles (k, x block); with two stages the next tile is
// fetched by asynchronous copies (landing in even/odd order) while the current
// one is transformed.
template <class T, int N>
__global__ void __launch_bounds__(ColCfg<T, N>::NTH)
    k_cols_dct_fdi(int nx, int nk, c_t<T>* __restrict__ S, Tabs<T> tb, SolveCoef co, const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    using Cfg = ColCfg<T, N>;
    constexpr int CW = Cfg::CW, NTH = Cfg::NTH, STAGES = Cfg::STAGES;
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* bufs = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x;
    const int nxb = (nx + CW - 1) / CW;
    const int ntiles = nk * nxb;
    auto stage = [&](int t, C* buf) {
        const int k = t / nxb, x0 = (t % nxb) * CW;
        const C* slab = S + (size_t)k * N * nx;
        for (int e = tid; e < N * CW; e += NTH) {
            const int c = e % CW, y = e / CW;
            const int x = x0 + c;
            C* d = &buf[dct_pos(y, N) * CW + c];
            if (x < nx) cp_async_val<sizeof(C)>(d, slab + (size_t)y * nx + x);
            else *d = mkc(T(0), T(0));
        }
        cp_async_commit_grp();
    };
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    if (STAGES == 2) stage(blockIdx.x, bufs);
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        C* buf = bufs + (STAGES == 2 ? (it & 1) : 0) * (Cfg::TILE / sizeof(C));
        if constexpr (STAGES == 2) {
            if (t + gridDim.x < ntiles) {
                stage(t + gridDim.x, bufs + ((it + 1) & 1) * (Cfg::TILE / sizeof(C)));
                cp_async_wait_grp<1>();
            } else {
                cp_async_wait_grp<0>();
            }
        } else {
            stage(t, buf);
            cp_async_wait_grp<0>();
        }
        __syncthreads();
        const int k = t / nxb, x0 = (t % nxb) * CW;
        C* slab = S + (size_t)k * N * nx;
        smem_fft<C, N, -1, NTH, CW, CW, 1>(buf, tb.twy);
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
        __syncthreads();   // buf is refilled two tiles later
    }
}

// ---------------------------------------------------------------------------
// Columns, warp-per-column form (128 <= N <= 512): a tile of 16 columns sits
// in shared memory column-major, column c at c*N with its element y at
// swz(y) ^ c (conflict-free both for the row-wise copies in and out and for
// the FFT passes).  Warp c transforms column c alone (forward DCT, divide,
// inverse); the CTA synchronizes only after the tile lands and before it is
// written back.  Persistent CTAs prefetch the next tile by cp.async.
// ---------------------------------------------------------------------------
template <class T, int N> struct ColWCfg {
    static constexpr int CW = 16, NTH = 32 * CW;
    static constexpr size_t TILE = sizeof(c_t<T>) * (size_t)N * CW;
    static constexpr int STAGES = 2 * TILE <= 160 * 1024 ? 2 : 1;
    static constexpr size_t SMEM = STAGES * TILE;
    static constexpr int MINB = sizeof(T) == 4 && N <= 256 ? 2 : 1;   // 64 registers for two CTAs per SM
};
template <class T, int N>
constexpr bool cols_warp_ok = N >= 128 && N <= (sizeof(T) == 4 ? 512 : 256);

__device__ __forceinline__ int colw_pos(int c, int y) { return swz<1>(y) ^ c; }

template <class T, int N>
__global__ void __launch_bounds__(512, ColWCfg<T, N>::MINB) k_cols_dct_fdi_w(int nx, int nk, c_t<T>* __restrict__ S, Tabs<T> tb,
                                                        SolveCoef co, const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    using Cfg = ColWCfg<T, N>;
    constexpr int CW = Cfg::CW, NTH = Cfg::NTH, STAGES = Cfg::STAGES, NP = N / 2 + 1, PPL = (NP + 31) / 32;
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* bufs = reinterpret_cast<C*>(smem_raw);
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int nxb = (nx + CW - 1) / CW;
    const int ntiles = nk * nxb;
    // copy in: element e of the tile is row y = e / CW, column c = e % CW
    auto stage = [&](int t, C* buf) {
        const int k = t / nxb, x0 = (t % nxb) * CW;
        const C* slab = S + (size_t)k * N * nx;
        for (int e = tid; e < N * CW; e += NTH) {
            const int c = e % CW, y = e / CW;
            C* d = &buf[c * N + colw_pos(c, y)];
            if (x0 + c < nx) cp_async_val<sizeof(C)>(d, slab + (size_t)y * nx + x0 + c);
            else *d = mkc(T(0), T(0));
        }
        cp_async_commit_grp();
    };
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    if (STAGES == 2) stage(blockIdx.x, bufs);
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        C* buf = bufs + (STAGES == 2 ? (it & 1) : 0) * (Cfg::TILE / sizeof(C));
        if constexpr (STAGES == 2) {
            if (t + gridDim.x < ntiles) {
                stage(t + gridDim.x, bufs + ((it + 1) & 1) * (Cfg::TILE / sizeof(C)));
                cp_async_wait_grp<1>();
            } else {
                cp_async_wait_grp<0>();
            }
        } else {
            stage(t, buf);
            cp_async_wait_grp<0>();
        }
        __syncthreads();
        const int k = t / nxb, x0 = (t % nxb) * CW;
        const int c = warp, x = x0 + c;
        C* col = buf + c * N;
        // forward FFT of the even/odd reordering of the stored column (key c)
        warp_fft<C, N, -1, true, true>(col, tb.twy, lane, c);
        if (x < nx) {
            const T lx = tb.lamx[x];
#pragma unroll
            for (int kk = 0; kk < PPL; ++kk) {
                const int p = lane + 32 * kk, q = (N - p) % N;
                if (p < NP) {
                    const int sp = colw_pos(c, p), sq = colw_pos(c, q);
                    const C wp = tb.wy[p], wq = tb.wy[q];
                    C Xp, Xq;
                    dct_post(col[sp], col[sq], wp, wq, Xp, Xq);
                    Xp = cdiv(Xp, shift_den(tb, k, lx + tb.lamy[p], c2, c1));
                    Xq = cdiv(Xq, shift_den(tb, k, lx + tb.lamy[q], c2, c1));
                    dct_pre(p, Xp, Xq, wp, wq, Xp, Xq);
                    col[sp] = Xp;
                    col[sq] = Xq;
                }
            }
        }
        __syncwarp();
        warp_fft<C, N, +1>(col, tb.twy, lane, c);
        __syncthreads();
        // copy out, row by row (16 columns = one coalesced segment per row)
        C* slab = S + (size_t)k * N * nx;
        const T inv = T(1) / T(N);
        for (int e = tid; e < N * CW; e += NTH) {
            const int cc = e % CW, y = e / CW;
            if (x0 + cc < nx) slab[(size_t)y * nx + x0 + cc] = scalec(buf[cc * N + colw_pos(cc, dct_pos(y, N))], inv);
        }
        __syncthreads();   // buf is refilled two tiles later
    }
}

// ---------------------------------------------------------------------------
// Columns, register four-step form (N = G*G, G = 8 or 16; FP32; nx even).  G
// lanes of a warp transform one column.  Write the column's even/odd
// reordered sequence as v_j, j = j1 + G j2.  Lane j1 takes the G-point DFT
// over j2 in registers and multiplies by exp(-2 pi i j1 k2 / N); the lanes
// swap through the column's shared-memory slot, after which lane k2 holds
// (Y_{j1,k2})_{j1}, whose G-point DFT over j1 is V_{k2 + G k1} in natural
// order.  The DCT-II coefficient pairs p with q = N - p, held by lane
// (G - k2) mod G: a shuffle brings V_q, each lane forms and divides its own
// X_p, a second shuffle brings the partner's X_q for the inverse
// pre-twiddle.  The inverse FFT runs the same steps backwards; its 1/N sits
// in the divide.
// Tile: CW = 16 columns as 8 column pairs; pair cp, reordered row r is the
// 16-byte chunk colr::chunk(N, cp, r) (an XOR swizzle within aligned groups
// of G chunks), so the copies in and out move 16 bytes per lane.  A half-warp holds 8 lanes of each column of a pair, so the
// strided lane accesses of both DFT steps cover all banks once.  Per-CTA
// tables in shared memory: the step twiddles as [j][s] (consecutive lanes,
// consecutive entries), the DCT twiddles w_p and the y eigenvalues.
// ---------------------------------------------------------------------------
template <class T, int N> struct ColRCfg {
    static constexpr int G = N == 64 ? 8 : 16;      // lanes per column = values per lane
    static constexpr int CW = 16, NPAIR = CW / 2, NTH = G * CW;
    static constexpr size_t TILE = sizeof(c_t<T>) * (size_t)N * CW;
    static constexpr int STAGES = 2;
    static constexpr size_t TAB_OFF = STAGES * TILE;
    static constexpr size_t SMEM = TAB_OFF + sizeof(c_t<T>) * (G * G + N) + sizeof(T) * N;
    static constexpr int MINB = N == 64 ? 8 : 2;
};
template <class T, int N>
constexpr bool cols_reg_ok = sizeof(T) == 4 && (N == 64 || N == 256);

// a * exp(DIR 2 pi i M / 16), M a compile-time constant
template <int DIR, int M, class C> __device__ __forceinline__ C rot16(C a) {
    using R = typename real_of<C>::type;
    constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173, h = 0.70710678118654752440;
    constexpr double cs[10] = {1.0, c1, h, s1, 0.0, -s1, -h, -c1, -1.0, -c1};
    constexpr double sn[10] = {0.0, s1, h, c1, 1.0, c1, h, s1, 0.0, -s1};
    if constexpr (M == 0) {
        return a;
    } else if constexpr (M == 4) {
        return rot90<DIR>(a);
    } else {
        const R c = R(cs[M]), s = R(DIR * sn[M]);
        return mkc(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}
// 16-point DFT in registers, natural order in and out: with j = a + 4c and
// k = b + 4d, X_k = sum_a w16^{ab} w4^{ad} (sum_c v_{a+4c} w4^{cb}).
template <int DIR, class C> __device__ __forceinline__ void dft16(C* v) {
    C t[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        t[a][0] = v[a];
        t[a][1] = v[a + 4];
        t[a][2] = v[a + 8];
        t[a][3] = v[a + 12];
        dft4<DIR>(t[a]);
    }
    t[1][1] = rot16<DIR, 1>(t[1][1]);
    t[1][2] = rot16<DIR, 2>(t[1][2]);
    t[1][3] = rot16<DIR, 3>(t[1][3]);
    t[2][1] = rot16<DIR, 2>(t[2][1]);
    t[2][2] = rot16<DIR, 4>(t[2][2]);
    t[2][3] = rot16<DIR, 6>(t[2][3]);
    t[3][1] = rot16<DIR, 3>(t[3][1]);
    t[3][2] = rot16<DIR, 6>(t[3][2]);
    t[3][3] = rot16<DIR, 9>(t[3][3]);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        C u[4] = {t[0][b], t[1][b], t[2][b], t[3][b]};
        dft4<DIR>(u);
        v[b] = u[0];
        v[b + 4] = u[1];
        v[b + 8] = u[2];
        v[b + 12] = u[3];
    }
}
template <int G, int DIR, class C> __device__ __forceinline__ void dft_reg(C* v) {
    if constexpr (G == 8) dft8<DIR>(v);
    else dft16<DIR>(v);
}
template <class C> __device__ __forceinline__ C shfl_c(C a, int src) {
    return mkc(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// approximate reciprocal (PTX rcp.approx.ftz.f32): its error is far below the
// rounding of the complex64 transforms around the divide
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// One step of the pair solve on the entries v[m] and v[G-1-m] of lane s,
// which holds V_{s + G k1} in v[k1].  For s != 0 the pair of entry m is the
// partner lane's entry G-1-m and vice versa; lane 0 is its own partner with
// pairs (k1, G - k1), so it takes entries m+1 and G-1-m here (m = G/2 - 1
// gives it the self-paired entry G/2) and keeps entry 0 for the end.  Each
// entry is updated in place exactly once.  Each lane forms its own scaled
// DCT-II coefficient X'_p = (w_p V_p + conj(w_p) V_q) dinv(p), dinv(p) =
// 1/(2 N D_p), and the inverse pre-twiddle V'_p = conj(w_p)(X'_p - i X'_q)
// takes the partner's X'_q as the partner rounded it, so both members of a
// pair are built from the same two coefficients: a rounding error of a small
// coefficient (cancellation when the other member dominates) stays in that
// coefficient's own mode instead of leaking into the other one, where the
// next residual would multiply it by the other, possibly far larger, D.
template <int G, int M, class C, class DenF>
__device__ __forceinline__ void pair_step(C* v, int s, int partner, const C* wt, DenF&& dinv) {
    constexpr int B = colr::pair_b(G, M), M1 = colr::pair_a_lane0(G, M);
    const bool z = s == 0;
    const C va = z ? v[M1] : v[M], vb = v[B];
    const int pa = s + G * (z ? M1 : M), pb = s + G * B;
    const C rb = shfl_c(vb, partner), ra = shfl_c(v[M], partner);   // the partner's entries B and M
    const C qa = z ? vb : rb, qb = z ? va : ra;                     // V of the pair of a, of b
    const C wa = wt[pa], wb = wt[pb];
    const C xa = cmul(dinv(pa), cmul(wa, va) + cmul(conjc(wa), qa));
    const C xb = cmul(dinv(pb), cmul(wb, vb) + cmul(conjc(wb), qb));
    const C rxb = shfl_c(xb, partner), rxa = shfl_c(xa, partner);
    const C xqa = z ? xb : rxb, xqb = z ? xa : rxa;                 // X' of the pair of a, of b
    const C na = cmul(conjc(wa), xa - rot90<+1>(xqa)), nb = cmul(conjc(wb), xb - rot90<+1>(xqb));
    if constexpr (M1 != B) {
        v[M] = z ? v[M] : na;
        v[M1] = z ? na : v[M1];
        v[B] = nb;
    } else {                                                // lane 0: a and b are both entry G/2
        v[M] = z ? v[M] : na;
        v[B] = z ? na : nb;
    }
}
template <int G, int M> struct PairSteps {
    template <class C, class DenF>
    __device__ __forceinline__ static void run(C* v, int s, int partner, const C* wt, DenF&& f) {
        pair_step<G, M>(v, s, partner, wt, f);
        PairSteps<G, M + 1>::run(v, s, partner, wt, f);
    }
};
template <int G> struct PairSteps<G, G / 2> {
    template <class C, class DenF>
    __device__ __forceinline__ static void run(C*, int, int, const C*, DenF&&) {}
};

template <class T, int N>
__global__ void __launch_bounds__(ColRCfg<T, N>::NTH, ColRCfg<T, N>::MINB)
    k_cols_dct_fdi_r(int nx, int nk, c_t<T>* __restrict__ S, Tabs<T> tb, SolveCoef co, const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    using Cfg = ColRCfg<T, N>;
    constexpr int G = Cfg::G, CW = Cfg::CW, NPAIR = Cfg::NPAIR, NTH = Cfg::NTH;
    constexpr int RSTEP = NTH / NPAIR, NCOPY = N / RSTEP;   // rows per copy sweep, sweeps per tile
    static_assert(G * G == N && (G == 8 || G == 16) && Cfg::STAGES == 2 && N % RSTEP == 0, "four-step shape");
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* chunks = reinterpret_cast<float4*>(smem_raw);   // TCH chunks per stage
    constexpr int TCH = (int)(Cfg::TILE / 16);
    C* tw1 = reinterpret_cast<C*>(smem_raw + Cfg::TAB_OFF);  // [j][s]: exp(-2 pi i s j / N)
    C* wt = tw1 + G * G;                                     // [p]: w_p = exp(-i pi p / (2N))
    T* ly = reinterpret_cast<T*>(wt + N);                    // [p]: y eigenvalues
    const int tid = threadIdx.x;
    const colr::Lane ln = colr::lane(G, tid);
    const int s = ln.s, half = ln.half, cp = ln.cp, c = ln.c, partner = ln.partner;
    const int nxb = (nx + CW - 1) / CW;
    const int ntiles = nk * nxb;
    // copies: thread (pair ccp, row y0 + RSTEP i) moves one 16-byte chunk
    const int ccp = tid % NPAIR, y0 = tid / NPAIR;
    auto chunk_of = [](int pr, int r) { return colr::chunk(N, pr, r); };
    auto stage = [&](int t, float4* buf) {
        const int k = t / nxb, x0 = (t % nxb) * CW;
        const bool ok = x0 + 2 * ccp < nx;
        const C* src = S + (size_t)k * N * nx + (size_t)y0 * nx + x0 + 2 * ccp;
#pragma unroll
        for (int i = 0; i < NCOPY; ++i) {
            const int y = y0 + RSTEP * i;
            float4* d = buf + chunk_of(ccp, dct_pos(y, N));
            if (ok) cp_async16(d, src + (size_t)RSTEP * i * nx);
            else *d = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_commit_grp();
    };
    stage(blockIdx.x, chunks);
    for (int i = tid; i < G * G; i += NTH) tw1[i] = tb.twy[(i / G) * (i % G)];
    for (int p = tid; p < N; p += NTH) {
        wt[p] = tb.wy[p];
        ly[p] = tb.lamy[p];
    }
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    const T sigma = T(0.5) / T(N);
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        float4* buf = chunks + (it & 1) * TCH;
        if (t + gridDim.x < ntiles) {
            stage(t + gridDim.x, chunks + ((it + 1) & 1) * TCH);
            cp_async_wait_grp<1>();
        } else {
            cp_async_wait_grp<0>();
        }
        __syncthreads();
        const int k = t / nxb, x0 = (t % nxb) * CW, x = x0 + c;
        C* el = reinterpret_cast<C*>(buf) + half;             // element r of our column: el[2 * chunk_of(cp, r)]
        C v[G];
        // forward: lane s = j1 transforms over j2, twiddles, swaps; then lane s = k2 over j1
#pragma unroll
        for (int j = 0; j < G; ++j) v[j] = el[2 * chunk_of(cp, s + G * j)];
        dft_reg<G, -1>(v);
#pragma unroll
        for (int j = 1; j < G; ++j) v[j] = cmul(v[j], tw1[j * G + s]);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < G; ++j) el[2 * chunk_of(cp, j + G * s)] = v[j];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < G; ++j) v[j] = el[2 * chunk_of(cp, s + G * j)];
        dft_reg<G, -1>(v);                                    // v[k1] = V_{s + G k1}
        // the solve on the FFT values (identity above); dead columns pass through
        const bool live = x < nx;
        const T lx = live ? tb.lamx[x] : T(0);
        const C l1 = tb.lam1[k], l2 = tb.lam2[k];
        // PinT-II adds lambda_3k Lam, lambda_3k = 1 - dt lambda_1k (zero otherwise)
        const T g3 = tb.dte != T(0) ? T(1) - tb.dte * l1.x : T(0), h3 = -tb.dte * l1.y;
        auto dinv = [&](int p) {
            const T lam = lx + ly[p];
            const T mu = (c2 * lam + c1) * lam;
            const T dx = fmaf(l2.x, mu, fmaf(g3, lam, l1.x)), dy = fmaf(l2.y, mu, fmaf(h3, lam, l1.y));
            const T m = sigma * rcp_approx(fmaf(dx, dx, dy * dy));
            return live ? mkc(dx * m, -dy * m) : mkc(sigma, T(0));
        };
        PairSteps<G, 0>::run(v, s, partner, wt, dinv);
        if (s == 0) v[0] = scalec(cmul(v[0], dinv(0)), T(2));  // p = 0 pairs with itself: V'_0 = X'_0
        // inverse: lane s = k2 over k1, twiddles, swaps; then lane s = j1 over k2
        dft_reg<G, +1>(v);
#pragma unroll
        for (int j = 1; j < G; ++j) v[j] = cmul(v[j], conjc(tw1[j * G + s]));
        __syncwarp();
#pragma unroll
        for (int j = 0; j < G; ++j) el[2 * chunk_of(cp, j + G * s)] = v[j];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < G; ++j) v[j] = el[2 * chunk_of(cp, s + G * j)];
        dft_reg<G, +1>(v);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < G; ++j) el[2 * chunk_of(cp, s + G * j)] = v[j];
        __syncthreads();
        // copy out: 16-byte chunks, row by row
        if (x0 + 2 * ccp < nx) {
            float4* dst = reinterpret_cast<float4*>(S + (size_t)k * N * nx + (size_t)y0 * nx + x0 + 2 * ccp);
#pragma unroll
            for (int i = 0; i < NCOPY; ++i)
                dst[(size_t)RSTEP * i * nx / 2] = buf[chunk_of(ccp, dct_pos(y0 + RSTEP * i, N))];
        }
        __syncthreads();   // buf is refilled two tiles later
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
// Fused 2-D solve of one frequency slice (square N x N grid, cosine path): a
// thread-block cluster of N/RB CTAs holds the slice in shared memory, CTA r
// owning rows RB*r .. RB*r+RB-1 and, after a transpose through distributed
// shared memory, the same range of columns.  Per slice: x forward -> transpose -> y
// forward, divide, y inverse -> transpose back -> x inverse.  The slice is read
// from and written to memory once (instead of three passes).
// ---------------------------------------------------------------------------
template <class T, int N> struct SliceCfg {
    static constexpr int RB = 32;               // rows (and columns) per CTA
    static constexpr int CS = N / RB;           // cluster size
    static constexpr int NTH = 512;
    static constexpr size_t SMEM = sizeof(c_t<T>) * 2 * (size_t)RB * N;
};

template <class T, int N>
__global__ void __launch_bounds__(512) k_slice2d(c_t<T>* __restrict__ S, Tabs<T> tb, SolveCoef co,
                                                 const Ctl* __restrict__ ctl) {
    using C = c_t<T>;
    constexpr int RB = SliceCfg<T, N>::RB, CS = SliceCfg<T, N>::CS, NTH = SliceCfg<T, N>::NTH;
    if (ctl && ctl->status != ST_RUNNING) return;   // same decision in every CTA of the cluster
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int k = blockIdx.x / CS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* A = reinterpret_cast<C*>(smem_raw);      // [RB][N]: rows y0 .. y0+RB-1
    C* B = A + RB * N;                          // [N][RB]: columns x0 .. x0+RB-1
    C* slab = S + (size_t)k * N * N;
    const int y0 = rank * RB, x0 = rank * RB;
    const int tid = threadIdx.x;
    // rows: load with the even/odd reordering, forward FFT, post-twiddle -> X (natural order)
#pragma unroll 4
    for (int e = tid; e < RB * N; e += NTH) {
        const int r = e / N, i = e % N;
        A[r * N + dct_pos(i, N)] = slab[(size_t)(y0 + r) * N + i];
    }
    __syncthreads();
    smem_fft<C, N, -1, NTH, RB, 1, N>(A, tb.twx);
    for (int e = tid; e < RB * (N / 2 + 1); e += NTH) {
        const int r = e / (N / 2 + 1), p = e % (N / 2 + 1), q = (N - p) % N;
        C Xp, Xq;
        dct_post(A[r * N + p], A[r * N + q], tb.wx[p], tb.wx[q], Xp, Xq);
        A[r * N + p] = Xp;
        A[r * N + q] = Xq;
    }
    cluster.sync();
    // transpose in: B[pos(y)][c] = X(y, x0 + c), rows y held by CTA y / RB
#pragma unroll 4
    for (int e = tid; e < N * RB; e += NTH) {
        const int c = e % RB, y = e / RB;
        const C* Ar = cluster.map_shared_rank(A, y / RB);
        B[dct_pos(y, N) * RB + c] = Ar[(y % RB) * N + x0 + c];
    }
    cluster.sync();
    // columns: forward FFT, divide, inverse FFT
    smem_fft<C, N, -1, NTH, RB, RB, 1>(B, tb.twy);
    const T c2 = T(co.c2), c1 = solve_c1<T>(co, ctl);
    for (int e = tid; e < (N / 2 + 1) * RB; e += NTH) {
        const int c = e % RB, p = e / RB, q = (N - p) % N;
        const C wp = tb.wy[p], wq = tb.wy[q];
        C Xp, Xq;
        dct_post(B[p * RB + c], B[q * RB + c], wp, wq, Xp, Xq);
        const T lx = tb.lamx[x0 + c];
        Xp = cdiv(Xp, shift_den(tb, k, lx + tb.lamy[p], c2, c1));
        Xq = cdiv(Xq, shift_den(tb, k, lx + tb.lamy[q], c2, c1));
        C Vp, Vq;
        dct_pre(p, Xp, Xq, wp, wq, Vp, Vq);
        B[p * RB + c] = Vp;
        B[q * RB + c] = Vq;
    }
    __syncthreads();
    smem_fft<C, N, +1, NTH, RB, RB, 1>(B, tb.twy);
    cluster.sync();
    // transpose out: row y0 + r, column x from CTA x / RB (y un-reordered, 1/N of the y inverse)
    const T inv = T(1) / T(N);
#pragma unroll 4
    for (int e = tid; e < RB * N; e += NTH) {
        const int r = e / N, x = e % N;
        const C* Br = cluster.map_shared_rank(B, x / RB);
        A[r * N + x] = scalec(Br[dct_pos(y0 + r, N) * RB + (x % RB)], inv);
    }
    cluster.sync();   // every remote read of B is done before any CTA moves on or exits
    // rows: pre-twiddle, inverse FFT, un-reorder, 1/N
    for (int e = tid; e < RB * (N / 2 + 1); e += NTH) {
        const int r = e / (N / 2 + 1), p = e % (N / 2 + 1), q = (N - p) % N;
        C Vp, Vq;
        dct_pre(p, A[r * N + p], A[r * N + q], tb.wx[p], tb.wx[q], Vp, Vq);
        A[r * N + p] = Vp;
        A[r * N + q] = Vq;
    }
    __syncthreads();
    smem_fft<C, N, +1, NTH, RB, 1, N>(A, tb.twx);
#pragma unroll 4
    for (int e = tid; e < RB * N; e += NTH) {
        const int r = e / N, i = e % N;
        slab[(size_t)(y0 + r) * N + i] = scalec(A[r * N + dct_pos(i, N)], inv);
    }
}

template <class T, int N>
static cudaError_t slice2d_n(int nk, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl, cudaStream_t st) {
    constexpr int CS = SliceCfg<T, N>::CS;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nk * CS, 1, 1);
    cfg.blockDim = dim3(SliceCfg<T, N>::NTH, 1, 1);
    cfg.dynamicSmemBytes = SliceCfg<T, N>::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_slice2d<T, N>, S, tb, co, ctl);
}

// Whether a cluster of this kernel can be resident at all on the current device
// (asked once per kernel; a device that cannot place the cluster uses the
// three-pass path).
template <class T, int N>
static int slice2d_fits() {
    static int ok = -1;
    if (ok < 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(SliceCfg<T, N>::CS, 1, 1);
        cfg.blockDim = dim3(SliceCfg<T, N>::NTH, 1, 1);
        cfg.dynamicSmemBytes = SliceCfg<T, N>::SMEM;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = SliceCfg<T, N>::CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        ok = cudaOccupancyMaxActiveClusters(&n, k_slice2d<T, N>, &cfg) == cudaSuccess && n > 0;
        cudaGetLastError();
    }
    return ok;
}

// Fused slices are used for 64^2 and 128^2 grids, where one kernel measured
// about 2x (64^2) and 1.5x (128^2) faster than the three passes; at 256^2 the
// large clusters (1-3 CTAs per SM) made it slower than three passes.
int slice2d_supported(const Geo& g, int fft_x, int fft_y, int f32) {
    if (g.dim != 2 || fft_x != 1 || fft_y != 1 || g.nx != g.ny) return 0;
    switch (g.nx) {
        case 64: return f32 ? slice2d_fits<float, 64>() : slice2d_fits<double, 64>();
        case 128: return f32 ? slice2d_fits<float, 128>() : slice2d_fits<double, 128>();
        default: return 0;
    }
}

template <class T>
cudaError_t launch_slice2d(const Geo& g, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                           cudaStream_t st) {
    const int nk = g.nt / 2 + 1;
    switch (g.nx) {
        case 64: return slice2d_n<T, 64>(nk, S, tb, co, ctl, st);
        case 128: return slice2d_n<T, 128>(nk, S, tb, co, ctl, st);
        default: return cudaErrorInvalidValue;
    }
}
template cudaError_t launch_slice2d<float>(const Geo&, float2*, const Tabs<float>&, SolveCoef, const Ctl*,
                                           cudaStream_t);
template cudaError_t launch_slice2d<double>(const Geo&, double2*, const Tabs<double>&, SolveCoef, const Ctl*,
                                            cudaStream_t);

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Resident CTAs of a persistent kernel on the current device: SMs x CTAs per SM.
template <class K>
static int persistent_ctas(K kernel, int nth, size_t smem) {
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, nth, smem) != cudaSuccess || per < 1)
        return 0;
    return nsm * per;
}

// Looked up once (from the configure step, outside any stream capture).
template <class T, int N, int MODE>
static int rows_resident() {
    static const int r = persistent_ctas(k_rows_dct<T, N, MODE>, RowCfg<T, N>::NTH, RowCfg<T, N>::SMEM);
    return r;
}

template <class T, int N, int MODE>
static int rows_w_resident();
template <class T, int N>
static cudaError_t cfg_rows() {
    cudaError_t e;
    const int sm = (int)RowCfg<T, N>::SMEM;
    if ((e = cudaFuncSetAttribute(k_rows_dct<T, N, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_rows_dct<T, N, MODE_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_rows_dct<T, N, MODE_FDI>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_rows_dct<T, N, MODE_PACK>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if (rows_resident<T, N, MODE_FWD>() <= 0 || rows_resident<T, N, MODE_INV>() <= 0 ||
        rows_resident<T, N, MODE_FDI>() <= 0 || rows_resident<T, N, MODE_PACK>() <= 0)
        return cudaErrorInvalidConfiguration;
    if constexpr (rows_warp_ok<T, N>) {
        const int smw = (int)RowWCfg<T, N>::SMEM;
        if ((e = cudaFuncSetAttribute(k_rows_dct_w<T, N, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smw)))
            return e;
        if ((e = cudaFuncSetAttribute(k_rows_dct_w<T, N, MODE_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smw)))
            return e;
        if ((e = cudaFuncSetAttribute(k_rows_dct_w<T, N, MODE_FDI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smw)))
            return e;
        if (rows_w_resident<T, N, MODE_FWD>() <= 0 || rows_w_resident<T, N, MODE_INV>() <= 0 ||
            rows_w_resident<T, N, MODE_FDI>() <= 0)
            return cudaErrorInvalidConfiguration;
    }
    return cudaSuccess;
}
template <class T, int N>
static int cols_resident();
template <class T, int N>
static int cols_w_resident();
template <class T, int N>
static int cols_r_resident();
template <class T, int N>
static cudaError_t cfg_cols() {
    cudaError_t e = cudaFuncSetAttribute(k_cols_dct_fdi<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ColCfg<T, N>::SMEM);
    if (e != cudaSuccess) return e;
    if (cols_resident<T, N>() <= 0) return cudaErrorInvalidConfiguration;
    if constexpr (cols_reg_ok<T, N>) {
        if ((e = cudaFuncSetAttribute(k_cols_dct_fdi_r<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ColRCfg<T, N>::SMEM)))
            return e;
        if (cols_r_resident<T, N>() <= 0) return cudaErrorInvalidConfiguration;
    }
    if constexpr (cols_warp_ok<T, N>) {
        if ((e = cudaFuncSetAttribute(k_cols_dct_fdi_w<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)ColWCfg<T, N>::SMEM)))
            return e;
        if (cols_w_resident<T, N>() <= 0) return cudaErrorInvalidConfiguration;
    }
    return cudaSuccess;
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
    if ((e = cudaFuncSetAttribute(k_slice2d<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SliceCfg<T, 64>::SMEM)))
        return e;
    if ((e = cudaFuncSetAttribute(k_slice2d<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)SliceCfg<T, 128>::SMEM)))
        return e;
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
static int rows_w_resident() {
    static const int r = persistent_ctas(k_rows_dct_w<T, N, MODE>, RowWCfg<T, N>::NTH, RowWCfg<T, N>::SMEM);
    return r;
}

template <class T, int N, int MODE>
static cudaError_t rows_n(int nrows, int ny, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                          cudaStream_t st) {
    if constexpr (rows_warp_ok<T, N>) {
        using W = RowWCfg<T, N>;
        const int resident = rows_w_resident<T, N, MODE>();
        if (resident <= 0) return cudaErrorInvalidConfiguration;
        const int need = (nrows + W::WARPS - 1) / W::WARPS;
        const int grid = need < resident ? need : resident;
        launch_pdl(k_rows_dct_w<T, N, MODE>, dim3(grid), dim3(W::NTH), W::SMEM, st, nrows, ny, S, tb, co, ctl);
        return cudaSuccess;
    }
    using Cfg = RowCfg<T, N>;
    const int resident = rows_resident<T, N, MODE>();
    if (resident <= 0) return cudaErrorInvalidConfiguration;
    const int ntiles = (nrows + Cfg::ROWS - 1) / Cfg::ROWS;
    const int grid = ntiles < resident ? ntiles : resident;
    launch_pdl(k_rows_dct<T, N, MODE>, dim3(grid), dim3(Cfg::NTH), Cfg::SMEM, st, nrows, ny, S, tb, co, ctl,
               PackDst<T>{});
    return cudaSuccess;
}
template <class T, int N>
static cudaError_t pack_solve_n(int nt, const c_t<T>* S, c_t<T>* z, const LongSolve<T>& ls, const Ctl* ctl,
                                cudaStream_t st) {
    using Cfg = RowCfg<T, N>;
    const int resident = rows_resident<T, N, MODE_PACK>();
    if (resident <= 0) return cudaErrorInvalidConfiguration;
    const int nrows = nt / 2 + 1;
    const int ntiles = (nrows + Cfg::ROWS - 1) / Cfg::ROWS;
    const int grid = ntiles < resident ? ntiles : resident;
    const PackDst<T> pd{z, long_plan(nt), nt};
    k_rows_dct<T, N, MODE_PACK><<<grid, Cfg::NTH, Cfg::SMEM, st>>>(nrows, 1, const_cast<c_t<T>*>(S), *ls.tb, ls.co,
                                                                   ctl, pd);
    return cudaSuccess;
}
template <class T>
cudaError_t launch_long_pack_solve(int nt, const c_t<T>* S, c_t<T>* z, const LongSolve<T>& ls, const Ctl* ctl,
                                   cudaStream_t st) {
    cudaError_t e;
    switch (ls.nx) {
#define P_(N) case N: e = pack_solve_n<T, N>(nt, S, z, ls, ctl, st); break;
        P_(2) P_(4) P_(8) P_(16) P_(32) P_(64) P_(128) P_(256) P_(512) P_(1024) P_(2048) P_(4096)
#undef P_
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
template cudaError_t launch_long_pack_solve<float>(int, const float2*, float2*, const LongSolve<float>&, const Ctl*,
                                                   cudaStream_t);
template cudaError_t launch_long_pack_solve<double>(int, const double2*, double2*, const LongSolve<double>&,
                                                    const Ctl*, cudaStream_t);
template <class T, int MODE>
static cudaError_t rows_dct(int nx, int nrows, int ny, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                            cudaStream_t st) {
    switch (nx) {
#define R_(N) case N: return rows_n<T, N, MODE>(nrows, ny, S, tb, co, ctl, st);
        R_(2) R_(4) R_(8) R_(16) R_(32) R_(64) R_(128) R_(256) R_(512) R_(1024) R_(2048) R_(4096)
#undef R_
        default: return cudaErrorInvalidValue;
    }
}
template <class T, int N>
static int cols_resident() {
    static const int r = persistent_ctas(k_cols_dct_fdi<T, N>, ColCfg<T, N>::NTH, ColCfg<T, N>::SMEM);
    return r;
}
template <class T, int N>
static int cols_w_resident() {
    static const int r = persistent_ctas(k_cols_dct_fdi_w<T, N>, ColWCfg<T, N>::NTH, ColWCfg<T, N>::SMEM);
    return r;
}
template <class T, int N>
static int cols_r_resident() {
    static const int r = persistent_ctas(k_cols_dct_fdi_r<T, N>, ColRCfg<T, N>::NTH, ColRCfg<T, N>::SMEM);
    return r;
}
template <class T, int N>
static cudaError_t cols_n(int nx, int nk, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                          cudaStream_t st) {
    if constexpr (cols_reg_ok<T, N>) {
        using W = ColRCfg<T, N>;
        if (nx % 2 == 0 && reinterpret_cast<uintptr_t>(S) % 16 == 0) {   // 16-byte copies of column pairs
            const int resident = cols_r_resident<T, N>();
            if (resident <= 0) return cudaErrorInvalidConfiguration;
            const int ntiles = nk * ((nx + W::CW - 1) / W::CW);
            const int grid = ntiles < resident ? ntiles : resident;
            launch_pdl(k_cols_dct_fdi_r<T, N>, dim3(grid), dim3(W::NTH), W::SMEM, st, nx, nk, S, tb, co, ctl);
            return cudaSuccess;
        }
    }
    if constexpr (cols_warp_ok<T, N>) {
        using W = ColWCfg<T, N>;
        const int resident = cols_w_resident<T, N>();
        if (resident <= 0) return cudaErrorInvalidConfiguration;
        const int ntiles = nk * ((nx + W::CW - 1) / W::CW);
        const int grid = ntiles < resident ? ntiles : resident;
        launch_pdl(k_cols_dct_fdi_w<T, N>, dim3(grid), dim3(W::NTH), W::SMEM, st, nx, nk, S, tb, co, ctl);
        return cudaSuccess;
    }
    using Cfg = ColCfg<T, N>;
    const int resident = cols_resident<T, N>();
    if (resident <= 0) return cudaErrorInvalidConfiguration;
    const int ntiles = nk * ((nx + Cfg::CW - 1) / Cfg::CW);
    const int grid = ntiles < resident ? ntiles : resident;
    launch_pdl(k_cols_dct_fdi<T, N>, dim3(grid), dim3(Cfg::NTH), Cfg::SMEM, st, nx, nk, S, tb, co, ctl);
    return cudaSuccess;
}
template <class T>
static cudaError_t cols_dct(int nx, int ny, int nk, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                            cudaStream_t st) {
    switch (ny) {
#define C_(N) case N: return cols_n<T, N>(nx, nk, S, tb, co, ctl, st);
        C_(2) C_(4) C_(8) C_(16) C_(32) C_(64) C_(128) C_(256) C_(512) C_(1024)
#undef C_
        default: return cudaErrorInvalidValue;
    }
}
template <class T, int MODE>
static void dense(int axis, int nx, int ny, int nk, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                  cudaStream_t st) {
    const int n = axis == 0 ? nx : ny;
    const int nvec = axis == 0 ? nk * ny : nk * nx;
    k_dense<T, MODE><<<nvec, 128, 2 * n * sizeof(c_t<T>), st>>>(axis, nx, ny, nvec, S, tb, co, ctl);
}

// Sine path of one axis (k_dst.cu).
template <class T, int MODE, int AXIS>
cudaError_t dst_axis(int n, int nx, int ny, long nlines, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                     cudaStream_t st);

// Axis kinds (fft_x, fft_y): 1 = cosine FFT path, 2 = sine (DST-I) FFT path, 0 = dense.
template <class T>
cudaError_t launch_spatial_stage(int stage, const Geo& g, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, int fft_x,
                                 int fft_y, const Ctl* ctl, cudaStream_t st) {
    const int nk = g.nt / 2 + 1;
    const int ny = g.dim == 2 ? g.ny : 1;
    cudaError_t e = cudaSuccess;
    if (g.dim == 1) {
        if (stage != 0) return cudaSuccess;
        if (fft_x == 1) e = rows_dct<T, MODE_FDI>(g.nx, nk, 1, S, tb, co, ctl, st);
        else if (fft_x == 2) e = dst_axis<T, MODE_FDI, 0>(g.nx, g.nx, 1, nk, S, tb, co, ctl, st);
        else dense<T, MODE_FDI>(0, g.nx, 1, nk, S, tb, co, ctl, st);
    } else if (stage == 0) {
        if (fft_x == 1) e = rows_dct<T, MODE_FWD>(g.nx, nk * ny, ny, S, tb, co, ctl, st);
        else if (fft_x == 2) e = dst_axis<T, MODE_FWD, 0>(g.nx, g.nx, ny, (long)nk * ny, S, tb, co, ctl, st);
        else dense<T, MODE_FWD>(0, g.nx, ny, nk, S, tb, co, ctl, st);
    } else if (stage == 1) {
        if (fft_y == 1) e = cols_dct<T>(g.nx, ny, nk, S, tb, co, ctl, st);
        else if (fft_y == 2) e = dst_axis<T, MODE_FDI, 1>(ny, g.nx, ny, (long)nk * g.nx, S, tb, co, ctl, st);
        else dense<T, MODE_FDI>(1, g.nx, ny, nk, S, tb, co, ctl, st);
    } else {
        if (fft_x == 1) e = rows_dct<T, MODE_INV>(g.nx, nk * ny, ny, S, tb, co, ctl, st);
        else if (fft_x == 2) e = dst_axis<T, MODE_INV, 0>(g.nx, g.nx, ny, (long)nk * ny, S, tb, co, ctl, st);
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
