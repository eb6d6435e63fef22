// k_residual_ff.cu - the all-at-once residual in float-float arithmetic (about
// 48 significant bits on the FP32 pipes) for the PINT_MIXED_FF precision, plus
// the conversions between FP64 and float-float iterates.
//
// Same operator and boundary treatment as k_residual.cu (Eq. 2.6 / 4.8 with
// alpha = 0; theta = 1 below, theta = 1/2 adds A(u_{n-1}), Eyre's splitting
// takes the Laplacian term at u_{n-1}):
//   r_n = (u_{n-1} - u_n)/dt - [c2 Lap^2 u_n + c1 Lap u_n + cN Lap(u_n^3)],
// evaluated as dt r_n (see k_residual_ff below).
// The stencil sums are error-free in their high words (a TwoSum chain), so the
// cancellation in the differences of smooth data is resolved to a few 2^-48 of
// the terms, the same order as the rounding of the stored iterate.  Output: s = gamma_n r_n rounded to FP32 (the alpha-scaled input of
// Step 1), and per-CTA partial sums of r^2 and u^2.
#include "ff.cuh"
#include "pint_common.cuh"
#include "pint_kernels.h"
#include "tma.cuh"

namespace pint {

__device__ __forceinline__ ff ext_read_ff(const ff* __restrict__ u, int gx, int gy, int nx, int ny, int dim,
                                          int bc) {
    float sgn = 1.f;
    if (bc == 1) {
        if (gx < 0) gx = -1 - gx;
        else if (gx >= nx) gx = 2 * nx - 1 - gx;
        if (dim == 2) {
            if (gy < 0) gy = -1 - gy;
            else if (gy >= ny) gy = 2 * ny - 1 - gy;
        }
    } else if (bc == 2) {
        if (gx < 0) gx = -gx;
        else if (gx >= nx) gx = 2 * (nx - 1) - gx;
        if (dim == 2) {
            if (gy < 0) gy = -gy;
            else if (gy >= ny) gy = 2 * (ny - 1) - gy;
        }
    } else {
        if (gx == -1 || gx == nx) return ffmk(0.f, 0.f);
        if (gx < -1) { gx = -2 - gx; sgn = -sgn; }
        else if (gx > nx) { gx = 2 * nx - gx; sgn = -sgn; }
        if (dim == 2) {
            if (gy == -1 || gy == ny) return ffmk(0.f, 0.f);
            if (gy < -1) { gy = -2 - gy; sgn = -sgn; }
            else if (gy > ny) { gy = 2 * ny - gy; sgn = -sgn; }
        }
    }
    if (gx < 0 || gx >= nx || (dim == 2 && (gy < 0 || gy >= ny))) return ffmk(0.f, 0.f);
    ff v = u[(dim == 2 ? gy * nx : 0) + gx];
    return ffmk(sgn * v.x, sgn * v.y);
}

// (a + b) - 2c, accurate
__device__ __forceinline__ ff ff_d2(ff a, ff b, ff c) { return ff_add(ff_add(a, b), ff_scale2(c, -2.f)); }
__device__ __forceinline__ ff ff_cube(ff x) { return ff_mul(ff_mul(x, x), x); }

// CTA tile: TX x TY points, each thread owns PPT points (rows ty, ty + TY/PPT, ...).
template <int DIM> struct ResTileFF;
template <> struct ResTileFF<1> { static constexpr int TX = 512, TY = 1, PPT = 2; };
template <> struct ResTileFF<2> { static constexpr int TX = 32, TY = 16, PPT = 2; };

// SQ (square cells, hx == hy, and every 1-D grid): the stencil sums are taken
// unscaled (integer coefficients only) and the 1/h^2, 1/h^4 factors are folded
// into the coefficients c1/h^2, c2/h^4, cN/h^2.  Otherwise each axis is scaled
// by its own 1/h^2 before the sum.
// Sum of a few double-word terms: one exact TwoSum chain over the high words,
// with the chain's rounding errors and all low words gathered in one FP32
// accumulator, then renormalized.  Cheaper than chained double-word additions
// (38 vs 82 flops for five terms); its error is a few 2^-48 of the terms'
// magnitude, about the rounding already present in the stored iterate.
struct ff_acc {
    float s, e;
    __device__ __forceinline__ explicit ff_acc(ff a) : s(a.x), e(a.y) {}
    __device__ __forceinline__ void add(ff t) {
        const ff q = two_sum(s, t.x);
        s = q.x;
        e = __fadd_rn(e, __fadd_rn(q.y, t.y));
    }
    __device__ __forceinline__ ff get() const { return two_sum(s, e); }
};

// SQ (square cells, hx == hy, and every 1-D grid): the stencil sums are taken
// unscaled (integer coefficients only) and the 1/h^2, 1/h^4 factors are folded
// into the coefficients c1/h^2, c2/h^4, cN/h^2.  Otherwise each axis is scaled
// by its own 1/h^2 before the sum.
// ACC: chained accurate double-word additions, whose error is relative to the
// (cancelled) result; used for very stiff problems, where the stencil terms
// exceed the result by many orders and the cheaper sum's error (relative to
// the terms) would dominate the residual.
template <int DIM, bool SQ, bool ACC>
__device__ __forceinline__ ff lap_ff(const ff* __restrict__ a, int c, int sx, const GeoFF& g) {
    if constexpr (SQ && ACC) {
        ff v = ff_add(a[c - 1], a[c + 1]);
        if constexpr (DIM == 2) {
            v = ff_add(v, a[c - sx]);
            v = ff_add(v, a[c + sx]);
        }
        return ff_add(v, ff_scale2(a[c], DIM == 2 ? -4.f : -2.f));
    } else if constexpr (SQ) {
        ff_acc acc(a[c - 1]);
        acc.add(a[c + 1]);
        if constexpr (DIM == 2) {
            acc.add(a[c - sx]);
            acc.add(a[c + sx]);
        }
        acc.add(ff_scale2(a[c], DIM == 2 ? -4.f : -2.f));
        return acc.get();
    } else {
        ff v = ff_mul(ff_d2(a[c - 1], a[c + 1], a[c]), g.ihx2);
        if constexpr (DIM == 2) v = ff_add(v, ff_mul(ff_d2(a[c - sx], a[c + sx], a[c]), g.ihy2));
        return v;
    }
}

// Neumann reflection of a halo index g in [-2, n+1] into [0, n): even about
// the cell faces (bc 1, cell-centred) or about the end vertices (bc 2).
__device__ __forceinline__ int reflect_n(int g, int n, int bc) {
    if (bc == 2) g = g < 0 ? -g : (g >= n ? 2 * (n - 1) - g : g);
    else g = g < 0 ? -1 - g : (g >= n ? 2 * n - 1 - g : g);
    return min(max(g, 0), n - 1);
}

// 8-byte asynchronous copy global -> shared (cp.async, cached in L1 for the
// halo overlap between neighbouring tiles), committed as one group per level.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The residual is computed scaled by dt,
//   r'_n = (u_{n-1} - u_n) - [c2' Lap^2 u_n + c1' Lap u_n + cN' Lap(u_n^3)],  c' = dt c,
// so the time difference needs no product; s = (gamma_n / dt) r' and the norm
// partials carry the factor 1/dt^2.  The CTA stages time level n+1 of its tile
// (with halo) by asynchronous copies while it computes level n.
template <int DIM, bool SQ, bool ACC, bool USEP>
__global__ void __launch_bounds__(256, 5) k_residual_ff(GeoFF g, const ff* __restrict__ U, const ff* __restrict__ u0,
                                                     const float* __restrict__ gamf, float* __restrict__ s_out,
                                                     double* __restrict__ partials, const Ctl* __restrict__ ctl,
                                                     int chunk) {
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    constexpr int TX = ResTileFF<DIM>::TX, TY = ResTileFF<DIM>::TY, PPT = ResTileFF<DIM>::PPT;
    constexpr int NTHR = TX * TY / PPT;
    constexpr int RSTEP = DIM == 2 ? TY / PPT : 0;     // row offset between a thread's points (2-D)
    constexpr int XSTEP = DIM == 2 ? 0 : TX / PPT;     // column offset (1-D)
    constexpr int HY = DIM == 2 ? 2 : 0;
    constexpr int SX = TX + 4, SY = TY + 2 * HY;
    constexpr int LX = TX + 2, LY = TY + (DIM == 2 ? 2 : 0);
    __shared__ __align__(16) ff su[2][SY * SX];
    __shared__ ff sL[LY * LX];
    __shared__ ff sW[LY * LX];   // u^3 (Cahn-Hilliard)
    __shared__ double red[2][NTHR / 32];

    const int tid = threadIdx.x;
    const int tx = tid % (DIM == 2 ? TX : TX / PPT), ty = tid / (DIM == 2 ? TX : TX / PPT);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(g.nt, n0 + chunk);
    const bool ch = g.cN.x != 0.f;
    const bool lin1 = g.c1.x != 0.f;
    const bool interior = x0 >= 2 && x0 + TX + 2 <= g.nx && (DIM == 1 || (y0 >= 2 && y0 + TY + 2 <= g.ny));
    // halo values are plain (reflected) copies except on simply supported boundary tiles
    const bool async_ok = interior || ((g.bc == 1 && g.nx >= 2 && (DIM == 1 || g.ny >= 2)) ||
                                       (g.bc == 2 && g.nx >= 3 && (DIM == 1 || g.ny >= 3)));

    // Per-thread work assignments, fixed for all levels (linear in the thread
    // index, so only the last warps of a pass idle): halo-tile elements
    // e = tid + a*NTHR of the staging copy, Laplacian points of the first pass.
    constexpr int NST = (SX * SY + NTHR - 1) / NTHR, NLP = (LX * LY + NTHR - 1) / NTHR;
    int goff[NST], soff[NST];            // source offset inside a level (-1: none), shared offset
#pragma unroll
    for (int a = 0; a < NST; ++a) {
        const int e = tid + a * NTHR;
        const int iy = e / SX, ix = e % SX;
        goff[a] = -1;
        soff[a] = e;
        if (e < SX * SY) {
            const int gy = DIM == 2 ? (interior ? y0 - HY + iy : reflect_n(y0 - HY + iy, g.ny, g.bc)) : 0;
            const int gx = interior ? x0 - 2 + ix : reflect_n(x0 - 2 + ix, g.nx, g.bc);
            goff[a] = gy * g.nx + gx;
        }
    }
    int lc[NLP];                          // su index of the point (-1: none); its sL index is tid + a*NTHR
#pragma unroll
    for (int a = 0; a < NLP; ++a) {
        const int e = tid + a * NTHR;
        lc[a] = e < LX * LY ? (DIM == 2 ? (e / LX + 1) * SX : 0) + e % LX + 1 : -1;
    }
    auto stage = [&](int n, ff* dst) {
        const ff* un = n < 0 ? u0 : U + (size_t)n * g.nspace;   // level -1 is the initial condition
        if (async_ok) {
#pragma unroll
            for (int a = 0; a < NST; ++a)
                if (goff[a] >= 0) cp_async8(&dst[soff[a]], un + goff[a]);
            cp_async_commit();
        } else {
            for (int e = tid; e < SX * SY; e += NTHR)
                dst[e] = ext_read_ff(un, x0 - 2 + e % SX, y0 - HY + e / SX, g.nx, g.ny, DIM, g.bc);
        }
    };

    int cu[PPT], cl[PPT];
    bool inside[PPT];
    ff uprev[PPT];
    float* sp[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int lx = tx + q * XSTEP, ly = ty + q * RSTEP;
        const int gx = x0 + lx, gy = y0 + ly;
        inside[q] = gx < g.nx && (DIM == 1 || gy < g.ny);
        const int pidx = (DIM == 2 ? gy * g.nx : 0) + gx;
        cu[q] = (ly + HY) * SX + lx + 2;
        cl[q] = (DIM == 2 ? (ly + 1) * LX : 0) + lx + 1;
        uprev[q] = ffmk(0.f, 0.f);
        if (inside[q]) uprev[q] = n0 == 0 ? u0[pidx] : U[(size_t)(n0 - 1) * g.nspace + pidx];
        sp[q] = s_out + (size_t)n0 * g.nspace + pidx;
    }
    float acc_r2 = 0.f, acc_u2 = 0.f;
    const float sdt = g.inv_dt.x;
    // theta = 1/2: A'(u_{n-1}) per point; Eyre's splitting: Lap u_{n-1} per point;
    // both from one extra level before the chunk
    const bool expl = g.expl != 0;
    constexpr bool usep = USEP;   // theta = 1/2 or Eyre (a separate instantiation keeps the default path lean)
    ff Aprev[PPT], Lprev[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) Aprev[q] = Lprev[q] = ffmk(0.f, 0.f);
    const int nfirst = usep ? n0 - 1 : n0;

    if (n0 < n1) stage(nfirst, su[0]);
    for (int n = nfirst; n < n1; ++n) {
        const ff* cur = su[(n - nfirst) & 1];
        if (async_ok) cp_async_wait_all();
        __syncthreads();                                   // level n staged; level n-1 fully consumed
        if (n + 1 < n1) stage(n + 1, su[(n + 1 - nfirst) & 1]);
#pragma unroll
        for (int a = 0; a < NLP; ++a)
            if (lc[a] >= 0) {
                sL[tid + a * NTHR] = lap_ff<DIM, SQ, ACC>(cur, lc[a], SX, g);
                if (ch) sW[tid + a * NTHR] = ff_cube(cur[lc[a]]);
            }
        __syncthreads();
        if constexpr (usep) {
            // Crank-Nicolson: dt r = u_{n-1} - u_n - A'(u_n) - A'(u_{n-1}), A' = dt A / 2 (linear equations);
            // Eyre: dt r = u_{n-1} - u_n - dt (c2 Lap^2 u_n + cN Lap u_n^3) - dt c1 Lap u_{n-1}
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if (inside[q]) {
                    const ff L = sL[cl[q]];
                    const ff lapL = lap_ff<DIM, SQ, ACC>(sL, cl[q], LX, g);
                    ff A = ff_mul(lapL, g.c2);
                    if (lin1 && !expl) A = ff_add(A, ff_mul(L, g.c1));
                    if (ch) A = ff_add(A, ff_mul(lap_ff<DIM, SQ, ACC>(sW, cl[q], LX, g), g.cN));
                    if (n >= n0) {
                        const ff u = cur[cu[q]];
                        const ff B = expl ? ff_mul(Lprev[q], g.c1) : Aprev[q];
                        ff r;
                        if constexpr (SQ && !ACC) {
                            ff_acc acc(uprev[q]);
                            acc.add(ff_neg(u));
                            acc.add(ff_neg(A));
                            acc.add(ff_neg(B));
                            r = acc.get();
                        } else {
                            r = ff_sub(ff_sub(ff_sub(uprev[q], u), A), B);
                        }
                        *sp[q] = fmaf(gamf[n] * sdt, r.x, gamf[n] * sdt * r.y);
                        acc_r2 = fmaf(r.x, r.x, acc_r2);
                        acc_u2 = fmaf(u.x, u.x, acc_u2);
                        uprev[q] = u;
                    }
                    Aprev[q] = A;
                    Lprev[q] = L;
                }
                if (n >= n0) sp[q] += g.nspace;
            }
            continue;
        }
        const float gm = gamf[n] * sdt;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            if (inside[q]) {
                const ff L = sL[cl[q]];
                const ff u = cur[cu[q]];
                const ff lapL = lap_ff<DIM, SQ, ACC>(sL, cl[q], LX, g);
                ff r;
                if constexpr (SQ && !ACC) {
                    ff_acc acc(uprev[q]);
                    acc.add(ff_neg(u));
                    acc.add(ff_neg(ff_mul(lapL, g.c2)));
                    if (lin1) acc.add(ff_neg(ff_mul(L, g.c1)));
                    if (ch) acc.add(ff_neg(ff_mul(lap_ff<DIM, SQ, ACC>(sW, cl[q], LX, g), g.cN)));
                    r = acc.get();
                } else {
                    ff A = ff_mul(lapL, g.c2);
                    if (lin1) A = ff_add(A, ff_mul(L, g.c1));
                    if (ch) A = ff_add(A, ff_mul(lap_ff<DIM, SQ, ACC>(sW, cl[q], LX, g), g.cN));
                    r = ff_sub(ff_sub(uprev[q], u), A);
                }
                *sp[q] = fmaf(gm, r.x, gm * r.y);
                acc_r2 = fmaf(r.x, r.x, acc_r2);
                acc_u2 = fmaf(u.x, u.x, acc_u2);
                uprev[q] = u;
            }
            sp[q] += g.nspace;
        }
    }
    const double idt = (double)g.inv_dt.x + (double)g.inv_dt.y;
    double a = warp_sum((double)acc_r2) * (idt * idt), b = warp_sum((double)acc_u2);
    const int warp = tid / 32, lane = tid % 32;
    if (lane == 0) { red[0][warp] = a; red[1][warp] = b; }
    __syncthreads();
    if (tid == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < NTHR / 32; ++w) { A += red[0][w]; B += red[1][w]; }
        size_t cta = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[2 * cta] = A;
        partials[2 * cta + 1] = B;
    }
}

// ---------------------------------------------------------------------------
// Narrow 1-D grids (nx <= 256): a tile is TN consecutive time levels of the
// whole row (TN a multiple of the warp count, about 1024 points), staged one
// tile ahead by asynchronous copies.  Stage row j holds level n0-1+j (row 0
// is level n0-1, u0 for the first tile) with two ghost points on each side,
// filled from the row by the boundary condition's even / odd extension once
// the tile has landed; the Laplacian rows carry one ghost point per side,
// which equals the same extension of their own interior values for all
// three boundary conditions.  The stencils then read shared memory with no
// boundary test.  Each warp works on its own run of rows with no block
// barrier between the passes (Lap u of the row into a private buffer, its
// ghosts, then the residual).  The arithmetic per point, and the order of its
// sums, is that of k_residual_ff.  Persistent CTAs (grid-stride over tiles);
// one pair of norm partials each.
// ---------------------------------------------------------------------------
constexpr int kNarrowNx = 256;
constexpr int kNarrowThreads = 256;
constexpr int kNarrowWarps = kNarrowThreads / 32;
constexpr int kNarrowMaxTn = 64;
static int narrow_tn(int nx) {
    int tn = (1024 / nx + kNarrowWarps - 1) / kNarrowWarps * kNarrowWarps;
    return tn < kNarrowWarps ? kNarrowWarps : (tn > kNarrowMaxTn ? kNarrowMaxTn : tn);
}
// Rows of private buffer per warp: Lap u of the row, of the previous row (theta = 1/2, Eyre), u^3 (Cahn-Hilliard).
static int narrow_wrows(bool usep, bool ch) { return 1 + (usep ? 1 : 0) + (ch ? 1 : 0); }
static size_t narrow_smem(int nx, int tn, int wrows) {
    return sizeof(ff) * ((size_t)2 * (tn + 1) * (nx + 4) + (size_t)kNarrowWarps * wrows * (nx + 2));
}

// Value at index i in [-2, nx+1] of a row whose interior a[0..nx) is stored:
// the boundary condition's extension outside.
__device__ __forceinline__ ff row_ext(const ff* __restrict__ a, int i, int nx, int bc) {
    if (i >= 0 && i < nx) return a[i];
    if (bc == 1) return a[i < 0 ? -1 - i : 2 * nx - 1 - i];
    if (bc == 2) return a[i < 0 ? -i : 2 * (nx - 1) - i];
    if (i == -1 || i == nx) return ffmk(0.f, 0.f);
    const ff v = a[i < 0 ? -2 - i : 2 * nx - i];
    return ffmk(-v.x, -v.y);
}
// Unscaled 1-D Laplacian sum a[x-1] + a[x+1] - 2 a[x] (ghosts stored) in the summation order of lap_ff<1, true, ACC>.
template <bool ACC>
__device__ __forceinline__ ff lap_row(const ff* __restrict__ a, int x) {
    const ff l = a[x - 1], r = a[x + 1], c = a[x];
    if constexpr (ACC) {
        return ff_add(ff_add(l, r), ff_scale2(c, -2.f));
    } else {
        ff_acc acc(l);
        acc.add(r);
        acc.add(ff_scale2(c, -2.f));
        return acc.get();
    }
}

template <bool ACC, bool USEP>
__global__ void __launch_bounds__(kNarrowThreads, 2)
    k_residual_ff_narrow(GeoFF g, const ff* __restrict__ U, const ff* __restrict__ u0, const float* __restrict__ gamf,
                         float* __restrict__ s_out, double* __restrict__ partials, const Ctl* __restrict__ ctl, int tn,
                         int wrows) {
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nx = g.nx, bc = g.bc, rows = tn + 1;
    const int SXN = nx + 4, LXN = nx + 2;           // padded row lengths (stage: 2 ghosts, Laplacian: 1)
    ff* stg = reinterpret_cast<ff*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    ff* wbuf = stg + (size_t)2 * rows * SXN + (size_t)warp * wrows * LXN;
    ff* Lc = wbuf + 1;                              // Lap u of the current row (index 0 = x 0)
    ff* Lp = USEP ? wbuf + LXN + 1 : nullptr;       // Lap u of the previous row
    const bool ch = g.cN.x != 0.f;
    ff* Wr = ch ? wbuf + (size_t)(USEP ? 2 : 1) * LXN + 1 : nullptr;   // u^3 of the current row
    const bool lin1 = g.c1.x != 0.f;
    const bool expl = g.expl != 0;
    const float sdt = g.inv_dt.x;
    __shared__ double red[2][kNarrowWarps];
    float acc_r2 = 0.f, acc_u2 = 0.f;
    const int ntiles = (g.nt + tn - 1) / tn;
    const int rpw = tn / kNarrowWarps;     // rows per warp
    // one warp per staged row: the row's interior, at offset 2 of its padded slot
    auto stage = [&](int t, ff* dst) {
        const int n0 = t * tn;
        const int nrows = min(tn, g.nt - n0) + 1;
        for (int j = warp; j < nrows; j += kNarrowWarps) {
            const int lev = n0 - 1 + j;
            const ff* src = lev < 0 ? u0 : U + (size_t)lev * g.nspace;
            ff* d = dst + (size_t)j * SXN + 2;
            for (int x = lane; x < nx; x += 32) cp_async8(&d[x], src + x);
        }
        cp_async_commit();
    };
    // ghosts of a row from its interior (i = -2, -1, nx, nx+1)
    auto ghost2 = [&](ff* row, int k) {
        const int i = k < 2 ? k - 2 : nx + k - 2;
        row[i] = row_ext(row, i, nx, bc);
    };
    // Lap u of a staged row (interior) and its one ghost per side; the calling warp only
    auto lap_of = [&](const ff* ur, ff* L) {
        for (int x = lane; x < nx; x += 32) L[x] = lap_row<ACC>(ur, x);
        __syncwarp();
        if (lane < 2) {
            const int i = lane == 0 ? -1 : nx;
            L[i] = row_ext(L, i, nx, bc);
        }
        __syncwarp();
    };
    if (blockIdx.x < ntiles) stage(blockIdx.x, stg);
    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        ff* cur = stg + (size_t)(it & 1) * rows * SXN;
        if (t + (int)gridDim.x < ntiles) {
            stage(t + gridDim.x, stg + (size_t)((it + 1) & 1) * rows * SXN);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();                   // tile t is in shared memory
        const int n0 = t * tn;
        const int nlev = min(tn, g.nt - n0);
        for (int e = tid; e < (nlev + 1) * 4; e += kNarrowThreads) ghost2(cur + (size_t)(e >> 2) * SXN + 2, e & 3);
        __syncthreads();                   // ghosts in place
        const int jb = 1 + warp * rpw, je = min(jb + rpw, nlev + 1);
        if (USEP && jb < je) lap_of(cur + (size_t)(jb - 1) * SXN + 2, Lp);
        for (int j = jb; j < je; ++j) {
            const ff* uj = cur + (size_t)j * SXN + 2;
            const ff* uq = uj - SXN;
            if (ch) {
                for (int x = lane; x < nx; x += 32) Wr[x] = ff_cube(uj[x]);
                __syncwarp();
                if (lane < 2) {
                    const int i = lane == 0 ? -1 : nx;
                    Wr[i] = row_ext(Wr, i, nx, bc);
                }
            }
            lap_of(uj, Lc);
            const int n = n0 - 1 + j;
            const float gm = gamf[n] * sdt;
            float* srow = s_out + (size_t)n * g.nspace;
            for (int x = lane; x < nx; x += 32) {
                const ff u = uj[x], up = uq[x], L = Lc[x];
                const ff lapL = lap_row<ACC>(Lc, x);
                ff r;
                if constexpr (USEP) {
                    ff A = ff_mul(lapL, g.c2);
                    if (lin1 && !expl) A = ff_add(A, ff_mul(L, g.c1));
                    if (ch) A = ff_add(A, ff_mul(lap_row<ACC>(Wr, x), g.cN));
                    ff B;
                    if (expl) {
                        B = ff_mul(Lp[x], g.c1);
                    } else {
                        B = ff_mul(lap_row<ACC>(Lp, x), g.c2);
                        if (lin1) B = ff_add(B, ff_mul(Lp[x], g.c1));
                    }
                    if constexpr (!ACC) {
                        ff_acc acc(up);
                        acc.add(ff_neg(u));
                        acc.add(ff_neg(A));
                        acc.add(ff_neg(B));
                        r = acc.get();
                    } else {
                        r = ff_sub(ff_sub(ff_sub(up, u), A), B);
                    }
                } else if constexpr (!ACC) {
                    ff_acc acc(up);
                    acc.add(ff_neg(u));
                    acc.add(ff_neg(ff_mul(lapL, g.c2)));
                    if (lin1) acc.add(ff_neg(ff_mul(L, g.c1)));
                    if (ch) acc.add(ff_neg(ff_mul(lap_row<ACC>(Wr, x), g.cN)));
                    r = acc.get();
                } else {
                    ff A = ff_mul(lapL, g.c2);
                    if (lin1) A = ff_add(A, ff_mul(L, g.c1));
                    if (ch) A = ff_add(A, ff_mul(lap_row<ACC>(Wr, x), g.cN));
                    r = ff_sub(ff_sub(up, u), A);
                }
                srow[x] = fmaf(gm, r.x, gm * r.y);
                acc_r2 = fmaf(r.x, r.x, acc_r2);
                acc_u2 = fmaf(u.x, u.x, acc_u2);
            }
            __syncwarp();                  // Lc (and Wr) are rewritten for the next row
            if constexpr (USEP) {
                ff* tmp = Lp;
                Lp = Lc;
                Lc = tmp;
            }
        }
        __syncthreads();                   // the stage of tile t is refilled two tiles later
    }
    const double idt = (double)g.inv_dt.x + (double)g.inv_dt.y;
    double a2 = warp_sum((double)acc_r2) * (idt * idt), b2 = warp_sum((double)acc_u2);
    if (lane == 0) { red[0][warp] = a2; red[1][warp] = b2; }
    __syncthreads();
    if (tid == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < kNarrowWarps; ++w) { A += red[0][w]; B += red[1][w]; }
        partials[2 * blockIdx.x] = A;
        partials[2 * blockIdx.x + 1] = B;
    }
}

// Persistent grid of the narrow kernel: resident CTAs per SM at its shared memory use (at most 4).
static int narrow_grid(const Geo& g, int tn) {
    const size_t sm = narrow_smem(g.nx, tn, narrow_wrows(true, true));
    int per = (int)((220 * 1024) / (sm + 1024));
    per = per < 1 ? 1 : (per > 4 ? 4 : per);
    const long tiles = (g.nt + tn - 1) / tn;
    const long want = 152L * per;
    return (int)(tiles < want ? tiles : want);
}

cudaError_t configure_residual_ff() {
    const int sm = (int)narrow_smem(kNarrowNx, narrow_tn(kNarrowNx), narrow_wrows(true, true));
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_residual_ff_narrow<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_residual_ff_narrow<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    if ((e = cudaFuncSetAttribute(k_residual_ff_narrow<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    return cudaFuncSetAttribute(k_residual_ff_narrow<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

static bool narrow_1d(const Geo& g) { return g.dim == 1 && g.nx <= kNarrowNx; }

__global__ void k_f64_to_ff(const double* __restrict__ in, ff* __restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = ff_from_double(in[i]);
}
// Exact float -> double by rebuilding the bit pattern on the integer pipes
// (normal numbers and zero; subnormals, inf and NaN take the conversion
// instruction).  Leaves one FP64 addition per element for hi + lo.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) {
        if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)(unsigned long long)(b & 0x80000000u) << 32);
        return (double)f;
    }
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}

__global__ void k_ff_to_f64(const ff* __restrict__ in, double* __restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const ff v = in[i];
        out[i] = f2d_exact(v.x) + f2d_exact(v.y);
    }
}
__global__ void k_broadcast_ff(ff* __restrict__ U, const ff* __restrict__ u0, int nspace, int nt) {
    size_t total = (size_t)nspace * nt;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        U[i] = u0[i % nspace];
}

static int grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b > 4 * 152 * 8 ? 4 * 152 * 8 : (b < 1 ? 1 : b));
}

int residual_ff_grid(const Geo& g, int& gx, int& gy, int& gz, int& chunk) {
    if (narrow_1d(g)) {
        chunk = narrow_tn(g.nx);
        gx = narrow_grid(g, chunk);
        gy = gz = 1;
        return gx;
    }
    const int TX = g.dim == 2 ? ResTileFF<2>::TX : ResTileFF<1>::TX, TY = g.dim == 2 ? ResTileFF<2>::TY : 1;
    gx = (g.nx + TX - 1) / TX;
    gy = g.dim == 2 ? (g.ny + TY - 1) / TY : 1;
    const long tiles = (long)gx * gy;
    // one wave: 152 SMs x 5 resident CTAs (the kernel's launch bound), split over time
    long want = 760 / tiles;
    if (want < 1) want = 1;
    chunk = (int)((g.nt + want - 1) / want);
    if (chunk < 4) chunk = 4;
    if (chunk > g.nt) chunk = g.nt;
    gz = (g.nt + chunk - 1) / chunk;
    return gx * gy * gz;
}

void launch_residual_ff(const GeoFF& g, const Geo& g64, const ff* U, const ff* u0, const float* gamf, float* s,
                        double* partials, const Ctl* ctl, cudaStream_t st) {
    int gx, gy, gz, chunk;
    residual_ff_grid(g64, gx, gy, gz, chunk);
    dim3 grid(gx, gy, gz);
    const bool sq = g64.dim == 1 || g64.ihx2 == g64.ihy2;
    const bool acc = g.accurate != 0;
    const bool usep = g.half || g.expl;
    if (narrow_1d(g64)) {
        const int wrows = narrow_wrows(usep, g.cN.x != 0.f);
        const size_t sm = narrow_smem(g64.nx, chunk, wrows);
#define PINT_RFN(A, P) \
    launch_pdl(k_residual_ff_narrow<A, P>, dim3(gx), dim3(kNarrowThreads), sm, st, g, U, u0, gamf, s, partials, ctl, \
               chunk, wrows)
        if (acc) { if (usep) PINT_RFN(true, true); else PINT_RFN(true, false); }
        else { if (usep) PINT_RFN(false, true); else PINT_RFN(false, false); }
#undef PINT_RFN
        return;
    }
#define PINT_RFF(D, S, A)                                                                                      \
    do {                                                                                                       \
        if (usep) launch_pdl(k_residual_ff<D, S, A, true>, grid, dim3(256), 0, st, g, U, u0, gamf, s, partials, \
                             ctl, chunk);                                                                       \
        else launch_pdl(k_residual_ff<D, S, A, false>, grid, dim3(256), 0, st, g, U, u0, gamf, s, partials, ctl,  \
                        chunk);                                                                                  \
    } while (0)
    if (g.dim == 2) {
        if (sq) { if (acc) PINT_RFF(2, true, true); else PINT_RFF(2, true, false); }
        else PINT_RFF(2, false, false);
    } else {
        if (acc) PINT_RFF(1, true, true); else PINT_RFF(1, true, false);
    }
#undef PINT_RFF
}
void launch_f64_to_ff(const double* in, ff* out, size_t n, cudaStream_t st) {
    k_f64_to_ff<<<grid_for(n), 256, 0, st>>>(in, out, n);
}
void launch_ff_to_f64(const ff* in, double* out, size_t n, cudaStream_t st) {
    k_ff_to_f64<<<grid_for(n), 256, 0, st>>>(in, out, n);
}
void launch_broadcast_ff(ff* U, const ff* u0, int nspace, int nt, cudaStream_t st) {
    k_broadcast_ff<<<grid_for((size_t)nspace * nt), 256, 0, st>>>(U, u0, nspace, nt);
}

}  // namespace pint
