// k_residual_fx.cu - the all-at-once residual of the linear equations in
// block fixed point on the integer pipes, FP64-accurate, for PINT_MIXED.
//
// Residual (Eq. 2.6 with alpha = 0; theta-method of Eq. 2.5, theta = 1 or 1/2;
// Eq. 4.8 for Cahn-Hilliard, theta = 1), evaluated scaled by dt:
//   dt r_n = u_{n-1} - u_n - theta dt A(u_n) - (1 - theta) dt A(u_{n-1}),
//   A(u) = c2 Lap^2 u + c1 Lap u + cN Lap(u^3)
//   (biharmonic: c1 = 0; linearized CH: c1 = beta|beta|, c2 = eps^2; CH: c1 = 1, cN = -1),
// on square cells (and every 1-D grid), where h^2 Lap and h^4 Lap^2 have
// integer stencils.  Each time level of a CTA's tile (halo 2, boundary
// conditions as reflections, as in k_residual.cu) is converted from the FP64
// iterate to 64-bit integers in the tile's unit 2^(E-56), E the tile's
// largest binary exponent, so both Laplacian passes are exact integer sums.
// The products with dt c1/h^2, dt c2/h^4 and dt cN/h^2 use each coefficient's
// full 53-bit mantissa (fx.cuh); the terms are aligned to the largest one's
// unit and added exactly.  The cube u^3 is formed per point from the level's
// integers by two exact 128-bit products, each truncated to 2^-56 of its bound,
// and its Laplacian is again an exact integer sum.  The result is then scaled by gamma_n/dt (Step 1's
// alpha-scaling, again from the FP64 factor's full mantissa) and rounded once
// to FP32, the input of the complex64 time transform.  Per CTA, the partial
// sum of r^2 feeds the convergence check.
//
// ROUT (pint_residual): the residual itself is written in FP64 and its
// square summed in FP64.
#include <atomic>

#include "fx.cuh"
#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

template <int DIM> struct FxTile;
template <> struct FxTile<1> { static constexpr int TX = 512, TY = 1, PPT = 2; };
template <> struct FxTile<2> { static constexpr int TX = 32, TY = 16, PPT = 2; };
constexpr int kFxThreads = 256;
// Resident CTAs per SM the launch bounds guarantee (theta = 1/2 carries the
// previous level's two Laplacians per point and needs more registers).
template <bool HALF> struct FxBlocks { static constexpr int value = HALF ? 4 : 4; };

// Source of halo element (gx, gy) of a time level: its offset within the
// level, or -1 for a zero (simply supported boundary vertex, or beyond the
// grid); *neg = 1 when the reflection is odd.  Same rules as ext_read in
// k_residual.cu.
__device__ __forceinline__ int fx_src(int gx, int gy, int nx, int ny, int dim, int bc, uint32_t* neg) {
    uint32_t s = 0;
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
        if (gx == -1 || gx == nx) return -1;
        if (gx < -1) { gx = -2 - gx; s ^= 1u; }
        else if (gx > nx) { gx = 2 * nx - gx; s ^= 1u; }
        if (dim == 2) {
            if (gy == -1 || gy == ny) return -1;
            if (gy < -1) { gy = -2 - gy; s ^= 1u; }
            else if (gy > ny) { gy = 2 * ny - gy; s ^= 1u; }
        }
    }
    if (gx < 0 || gx >= nx || (dim == 2 && (gy < 0 || gy >= ny))) return -1;
    *neg = s << 31;
    return (dim == 2 ? gy * nx : 0) + gx;
}

// Unscaled Laplacian stencil (3 or 5 points) at index c of an integer tile with row stride sx.
template <int DIM>
__device__ __forceinline__ int64_t fx_lap(const int64_t* __restrict__ a, int c, int sx) {
    if constexpr (DIM == 2) return a[c - 1] + a[c + 1] + a[c - sx] + a[c + sx] - 4 * a[c];
    else return a[c - 1] + a[c + 1] - 2 * a[c];
}

// 2^k as the product of two floats in the normal range (k within +-252).
__device__ __forceinline__ void fx_pow2_pair(int k, float& f1, float& f2) {
    int k1 = k >> 1, k2 = k - k1;
    k1 = min(max(k1, -126), 127);
    k2 = min(max(k2, -126), 127);
    f1 = __int_as_float((k1 + 127) << 23);
    f2 = __int_as_float((k2 + 127) << 23);
}

// The work is the list of (tile, level) units, tile-major; CTA c of C takes the
// contiguous units [c U / C, (c+1) U / C), which may span the end of one tile's
// levels and the start of the next tile's: every CTA gets the same number of
// levels to within one, whatever the tile count.
template <int DIM, bool HALF, bool ROUT, bool CUBE>
__global__ void __launch_bounds__(kFxThreads, FxBlocks<HALF>::value)
    k_residual_fx(GeoFX g, const double* __restrict__ U, const double* __restrict__ u0,
                  const double* __restrict__ gdt, const float* __restrict__ igamf, float* __restrict__ s_out,
                  double* __restrict__ r_out, double* __restrict__ partials, const Ctl* __restrict__ ctl) {
    pdl_wait();
    if (ctl && ctl->status != ST_RUNNING) return;
    constexpr int TX = FxTile<DIM>::TX, TY = FxTile<DIM>::TY, PPT = FxTile<DIM>::PPT;
    constexpr int NTHR = kFxThreads, NW = NTHR / 32;
    static_assert((NW & (NW - 1)) == 0 && NW <= 32, "per-warp maxima are reduced by one warp");
    constexpr int RSTEP = DIM == 2 ? TY / PPT : 0, XSTEP = DIM == 2 ? 0 : TX / PPT;
    constexpr int HY = DIM == 2 ? 2 : 0;
    constexpr int SX = TX + 4, SY = TY + 2 * HY;
    constexpr int LX = TX + 2, LY = TY + (DIM == 2 ? 2 : 0);
    constexpr int NST = (SX * SY + NTHR - 1) / NTHR, NLP = (LX * LY + NTHR - 1) / NTHR;
    constexpr int L2GROW = DIM == 2 ? 3 : 2;     // |Lap L1| <= 8 max|L1| (2-D), 4 max|L1| (1-D)
    static_assert(!(CUBE && HALF), "the cubic term comes with theta = 1");
    __shared__ int64_t sfx[2][SY * SX];
    __shared__ int64_t sL[2][LY * LX];
    __shared__ int64_t scub[CUBE ? SY * SX : 1];   // u^3 in 2^(3E-56) (read before the level's second barrier)
    __shared__ int sbN[NW];
    __shared__ int smax[2][NW];
    __shared__ int smaxp[NW];
    __shared__ int sbL[NW], sbD[NW];
    __shared__ double red[NW], red2[NW];

    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int tx = tid % (DIM == 2 ? TX : TX / PPT), ty = tid / (DIM == 2 ? TX : TX / PPT);
    int lc[NLP];
#pragma unroll
    for (int a = 0; a < NLP; ++a) {
        const int e = tid + a * NTHR;
        lc[a] = e < LX * LY ? (DIM == 2 ? (e / LX + 1) * SX : 0) + e % LX + 1 : -1;
    }
    const int tiles_x = (g.nx + TX - 1) / TX;
    const long long units = (long long)tiles_x * (DIM == 2 ? (g.ny + TY - 1) / TY : 1) * g.nt;
    const long long ub = units * blockIdx.x / gridDim.x, ue = units * (blockIdx.x + 1) / gridDim.x;
    float acc = 0.f;
    double accd = 0.0, accu2 = 0.0;
    for (long long u = ub; u < ue;) {
        // one segment: levels n0 .. n1-1 of one tile
        const int tile = (int)(u / g.nt);
        const int n0 = (int)(u - (long long)tile * g.nt);
        const int n1 = (int)min((long long)g.nt, n0 + (ue - u));
        u += n1 - n0;
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        const int nfirst = HALF ? n0 - 1 : n0;
        // the previous segment's last level is done with the shared buffers
        __syncthreads();

        // staging map (fixed for the segment's levels): this thread loads elements tid + a NTHR
        int goff[NST];
        uint32_t gneg[NST];
#pragma unroll
        for (int a = 0; a < NST; ++a) {
            const int e = tid + a * NTHR;
            goff[a] = -1;
            gneg[a] = 0;
            if (e < SX * SY) goff[a] = fx_src(x0 - 2 + e % SX, y0 - HY + e / SX, g.nx, g.ny, DIM, g.bc, &gneg[a]);
        }
        uint32_t rhi[NST], rlo[NST];
        auto load = [&](int n) {
            const double* un = n < 0 ? u0 : U + (size_t)n * g.nspace;
#pragma unroll
            for (int a = 0; a < NST; ++a) {
                if (goff[a] >= 0) {
                    const unsigned long long v = __ldg(reinterpret_cast<const unsigned long long*>(un + goff[a]));
                    rhi[a] = (uint32_t)(v >> 32) ^ gneg[a];
                    rlo[a] = (uint32_t)v;
                } else {
                    rhi[a] = 0u;
                    rlo[a] = 0u;
                }
            }
        };
        auto expmax = [&]() {
            int f = 0;
#pragma unroll
            for (int a = 0; a < NST; ++a) f = max(f, fx_expfield(rhi[a]));
            return (int)__reduce_max_sync(0xffffffffu, (unsigned)f);
        };

        int cu[PPT], cl[PPT];
        bool inside[PPT];
        size_t po[PPT];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int lx = tx + q * XSTEP, ly = ty + q * RSTEP;
            const int gx = x0 + lx, gy = y0 + ly;
            inside[q] = gx < g.nx && (DIM == 1 || gy < g.ny);
            po[q] = (size_t)(DIM == 2 ? gy * g.nx : 0) + gx;
            cu[q] = (ly + HY) * SX + lx + 2;
            cl[q] = (DIM == 2 ? (ly + 1) * LX : 0) + lx + 1;
        }
        // previous level per point in the tile-uniform unit 2^(Ep-56) (theta = 1/2: with its two Laplacians)
        int64_t up[PPT], L1p[PPT], L2p[PPT];
        uint32_t uph[PPT], upl[PPT];
        int fp = 0;
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            up[q] = L1p[q] = L2p[q] = 0;
            uph[q] = upl[q] = 0u;
            if (!HALF && inside[q]) {
                const double* src = n0 == 0 ? u0 : U + (size_t)(n0 - 1) * g.nspace;
                const unsigned long long v = __ldg(reinterpret_cast<const unsigned long long*>(src + po[q]));
                uph[q] = (uint32_t)(v >> 32);
                upl[q] = (uint32_t)v;
                fp = max(fp, fx_expfield(uph[q]));
            }
        }
        if (n0 < n1) {
            load(nfirst);
            const int f = expmax();
            const int f2 = (int)__reduce_max_sync(0xffffffffu, (unsigned)fp);
            if (lane == 0) {
                smax[0][warp] = f;
                smaxp[warp] = f2;
            }
        }
        __syncthreads();
        int Ep = -958, bL1p = 0;
        if (!HALF) {
            int f = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) f = max(f, smaxp[w]);
            Ep = max(fx_tile_exp(f), -958);
#pragma unroll
            for (int q = 0; q < PPT; ++q) up[q] = fx_from_f64_fast(uph[q], upl[q], Ep);
        }
        for (int n = nfirst; n < n1; ++n) {
            const int b = (n - nfirst) & 1;
            // the warps' maxima: lane w reads warp w's, one redux over the warp
            const int fmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)smax[b][lane & (NW - 1)]);
            const bool bad = fmax == 0x7FF;   // an infinity or NaN in the tile
            const int E = max(fx_tile_exp(fmax), -958);
#pragma unroll
            for (int a = 0; a < NST; ++a)
                if (tid + a * NTHR < SX * SY) {
                    const int64_t v = fx_from_f64_fast(rhi[a], rlo[a], E);
                    sfx[b][tid + a * NTHR] = v;
                    if constexpr (CUBE) {
                        // |v| < 2^56: P = floor(v^2 / 2^56) < 2^56 in 2^(2E-56), C = floor(v P / 2^56) in 2^(3E-56)
                        const int64_t av = v < 0 ? -v : v;
                        scub[tid + a * NTHR] = fx_mul_shr(v, fx_mul_shr(av, av, 56), 56);
                    }
                }
            if (n + 1 < n1) load(n + 1);
            // level-uniform unit: both levels in 2^(Em-56)
            const int Em = max(E, Ep);
            const uint32_t dE = (uint32_t)(Em - E), dEp = (uint32_t)(Em - Ep);
            const bool same = dE == 0u && dEp == 0u;
            __syncthreads();
            // first Laplacian pass, with the tile's largest |L1| and |u_{n-1} - u_n| (as bit counts)
            // v ^ (v >> 63) is |v| or |v| - 1: the bits of the OR of those, plus one, bound every |v|
            uint64_t orl = 0, ord = 0;
#pragma unroll
            for (int a = 0; a < NLP; ++a)
                if (lc[a] >= 0) {
                    const int64_t v = fx_lap<DIM>(sfx[b], lc[a], SX);
                    sL[b][tid + a * NTHR] = v;
                    orl |= (uint64_t)(v ^ (v >> 63));
                }
            int64_t LC[PPT];   // Lap(u^3) at this thread's points (unscaled stencil, 2^(3E-56))
            uint64_t orn = 0;
            if (!(HALF && n < n0)) {
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    LC[q] = 0;
                    if (inside[q]) {
                        const int64_t un = sfx[b][cu[q]];
                        const int64_t D = same ? up[q] - un : fx_sar(up[q], dEp) - fx_sar(un, dE);
                        ord |= (uint64_t)(D ^ (D >> 63));
                        if constexpr (CUBE) {
                            LC[q] = fx_lap<DIM>(scub, cu[q], SX);
                            orn |= (uint64_t)(LC[q] ^ (LC[q] >> 63));
                        }
                    }
                }
            }
            int bl = orl ? 65 - fx_clz64(orl) : 0, bd = ord ? 65 - fx_clz64(ord) : 0;
            bl = (int)__reduce_max_sync(0xffffffffu, (unsigned)bl);
            bd = (int)__reduce_max_sync(0xffffffffu, (unsigned)bd);
            if (lane == 0) {
                sbL[warp] = bl;
                sbD[warp] = bd;
            }
            if constexpr (CUBE) {
                const int bn = (int)__reduce_max_sync(0xffffffffu, (unsigned)(orn ? 65 - fx_clz64(orn) : 0));
                if (lane == 0) sbN[warp] = bn;
            }
            if (n + 1 < n1) {
                const int f = expmax();
                if (lane == 0) smax[b ^ 1][warp] = f;
            }
            __syncthreads();
            const int bL1 = (int)__reduce_max_sync(0xffffffffu, (unsigned)sbL[lane & (NW - 1)]);
            const int bD = (int)__reduce_max_sync(0xffffffffu, (unsigned)sbD[lane & (NW - 1)]);
            if (HALF && n < n0) {
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    up[q] = sfx[b][cu[q]];
                    L1p[q] = sL[b][cl[q]];
                    L2p[q] = fx_lap<DIM>(sL[b], cl[q], LX);
                }
                Ep = E;
                bL1p = bL1;
                continue;
            }
            // Terms in the unit 2^(Q+Em-56) of the exact products L M: c2 L2, c1 L1 and D 2^-Q.  Their
            // largest magnitude in this tile, 2^emax, sets the output unit 2^X, X = Q + Em - 56 + S with
            // S = emax - 60 (>= 0): every term is then resolved to 2^-60 of the largest one.
            // bits of the Laplacian sums as used (a shift to the unit Em only lowers them)
            const int bL = HALF ? max(bL1, bL1p) + 1 : bL1;
            // (coefficient i enters as M_i 2^(Q - dQ_i); the cube's unit is 2^(3E-56) against 2^(Em-56))
            const int e2 = bL + L2GROW + g.bM2 - g.dQ2, e1 = bL + g.bM1 - g.dQ1, eD = bD - g.Q;
            int emax = max(e2, eD);
            if (g.lin1) emax = max(emax, e1);
            if constexpr (CUBE) {
                const int bN = (int)__reduce_max_sync(0xffffffffu, (unsigned)sbN[lane & (NW - 1)]);
                if (bN > 0) emax = max(emax, bN + g.bMN - g.dQN + 3 * E - Em);
            }
            const int S = max(emax - 60, 0);
            const int S2 = S + g.dQ2, S1 = S + g.dQ1, SN = S + g.dQN - (3 * E - Em);
            const int X = g.Q + Em - 56 + S;
            const int kD = -g.Q - S;                              // D 2^-Q in units 2^S
            float Gh = 0.f, Gl = 0.f, f1 = 0.f, f2 = 0.f, ig = 0.f;
            if (!ROUT) {
                // gamma_n / dt = (Gh + Gl) 2^(gex - 1046); the output is R 2^X gamma_n / dt
                int gex;
                fx_split_f64((uint64_t)__double_as_longlong(__ldg(gdt + n)), Gh, Gl, gex);
                fx_pow2_pair(X + gex - 1046, f1, f2);
                ig = __ldg(igamf + n);
            }
            float lu2 = 0.f;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                if (!inside[q]) continue;
                const int64_t un = sfx[b][cu[q]];
                const int64_t L1o = sL[b][cl[q]];
                const int64_t L2o = fx_lap<DIM>(sL[b], cl[q], LX);
                int64_t D, L1 = L1o, L2 = L2o;
                if (same) {
                    D = up[q] - un;
                } else {
                    D = fx_sar(up[q], dEp) - fx_sar(un, dE);
                    L1 = fx_sar(L1o, dE);
                    L2 = fx_sar(L2o, dE);
                }
                int64_t L1s = L1, L2s = L2;
                if constexpr (HALF) {
                    L1s += same ? L1p[q] : fx_sar(L1p[q], dEp);
                    L2s += same ? L2p[q] : fx_sar(L2p[q], dEp);
                }
                int64_t R = kD >= 0 ? (D << kD) : fx_sar(D, (uint32_t)(-kD));
                R -= fx_mul_shr(L2s, g.M2, S2);
                if (g.lin1) {
                    const int64_t t1 = fx_mul_shr(L1s, g.M1, S1);
                    R = g.neg1 ? R + t1 : R - t1;
                }
                if constexpr (CUBE) {
                    // SN < 0 only when |LC MN| < 2^(60 + SN): the low word is then the exact product
                    const int64_t tN = SN >= 0 ? fx_mul_shr(LC[q], g.MN, SN)
                                               : (int64_t)((uint64_t)LC[q] * (uint64_t)g.MN) << (uint32_t)(-SN);
                    R = g.negN ? R + tN : R - tN;
                    // sum u^2 for the mean Jacobian 3 mean(u^2): u = un 2^(E-56)
                    const float vf = fx_to_f32_pair(un, 1.f, 0.f, 1.f, 1.f);
                    lu2 = fmaf(vf, vf, lu2);
                }
                const size_t o = (size_t)n * g.nspace + po[q];
                if constexpr (ROUT) {
                    const double r = bad ? __longlong_as_double(0x7FF8000000000000ll) : ldexp((double)R, X) * g.inv_dt;
                    if (r_out) r_out[o] = r;
                    accd = fma(r, r, accd);
                } else {
                    const float sv = bad ? __int_as_float(0x7FC00000) : fx_to_f32_pair(R, Gh, Gl, f1, f2);
                    s_out[o] = sv;
                    const float rv = sv * ig;
                    acc = fmaf(rv, rv, acc);
                }
                up[q] = un;
                if constexpr (HALF) {
                    L1p[q] = L1o;
                    L2p[q] = L2o;
                }
            }
            if constexpr (CUBE) accu2 = fma((double)lu2, ldexp(1.0, 2 * E - 112), accu2);
            Ep = E;
            bL1p = bL1;
        }
    }
    // deterministic block reduction of sum r^2 and (Cahn-Hilliard) sum u^2
    double a = warp_sum(ROUT ? accd : (double)acc);
    const double a2 = CUBE ? warp_sum(accu2) : 0.0;
    if (lane == 0) {
        red[warp] = a;
        red2[warp] = a2;
    }
    __syncthreads();
    if (tid == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < NW; ++w) {
            A += red[w];
            B += red2[w];
        }
        partials[2 * blockIdx.x] = A;
        partials[2 * blockIdx.x + 1] = B;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Linear equations with theta = 1 or 1/2, and Cahn-Hilliard (PinT-I, theta = 1),
// on square cells or in 1-D.
int residual_fx_supported(const Geo& g) {
    if (g.expl || !(g.dim == 1 || g.ihx2 == g.ihy2)) return 0;
    if (g.cN != 0.0) return g.th == 1.0;
    return g.th == 1.0 || g.th == 0.5;
}

// Each coefficient c_i = theta dt c1/h^2, theta dt c2/h^4, theta dt cN/h^2
// (theta = 1/2 is exact) as its own 53-bit mantissa M_i and exponent:
// |c_i| = M_i 2^(Q - dQ_i), Q the largest coefficient's exponent.  The products
// L M_i are exact; the kernel picks per tile and level how many low bits of
// them to drop.
GeoFX make_geo_fx(const Geo& g) {
    GeoFX f{};
    f.nx = g.nx;
    f.ny = g.ny;
    f.dim = g.dim;
    f.bc = g.bc;
    f.nt = g.nt;
    f.nspace = g.nspace;
    f.half = g.th < 1.0 ? 1 : 0;
    f.inv_dt = g.inv_dt;
    const double c1 = g.th * g.dt * g.c1 * g.ihx2, c2 = g.th * g.dt * g.c2 * g.ihx2 * g.ihx2,
                 cN = g.th * g.dt * g.cN * g.ihx2;
    const double cs[3] = {c1, c2, cN};
    int q[3];
    int Q = -1000;
    for (int i = 0; i < 3; ++i) {
        int e = 0;
        if (cs[i] != 0.0) frexp(cs[i], &e);
        q[i] = cs[i] != 0.0 ? e - 53 : -100000;
        if (cs[i] != 0.0 && q[i] > Q) Q = q[i];
    }
    f.Q = Q;
    int64_t* M[3] = {&f.M1, &f.M2, &f.MN};
    int* bM[3] = {&f.bM1, &f.bM2, &f.bMN};
    int* dQ[3] = {&f.dQ1, &f.dQ2, &f.dQN};
    for (int i = 0; i < 3; ++i) {
        *M[i] = 0;
        *bM[i] = 0;
        *dQ[i] = 0;
        if (cs[i] == 0.0) continue;
        *dQ[i] = Q - q[i];
        *M[i] = (int64_t)llrint(ldexp(fabs(cs[i]), -q[i]));   // exact: the 53-bit mantissa
        for (int64_t t = *M[i]; t; t >>= 1) ++*bM[i];
    }
    f.lin1 = c1 != 0.0 ? 1 : 0;
    f.neg1 = c1 < 0.0 ? 1 : 0;
    f.cube = cN != 0.0 ? 1 : 0;
    f.negN = cN < 0.0 ? 1 : 0;
    return f;
}

// SMs of the current device (looked up once per device).
static int fx_sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = cached[dev].load(std::memory_order_relaxed);
    if (v < 1) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 152;
        cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// One resident wave (SMs x the CTAs per SM that the launch bounds guarantee),
// at least 4 levels per CTA.  gx = CTAs, gy = gz = 1, chunk = units per CTA
// (rounded up).  Returns the CTA count, which is also the number of partials.
int residual_fx_grid(const Geo& g, int& gx, int& gy, int& gz, int& chunk) {
    const int TX = g.dim == 2 ? FxTile<2>::TX : FxTile<1>::TX, TY = g.dim == 2 ? FxTile<2>::TY : 1;
    const long long tiles = (long long)((g.nx + TX - 1) / TX) * (g.dim == 2 ? (g.ny + TY - 1) / TY : 1);
    const long long units = tiles * g.nt;
    long long c = (long long)fx_sm_count() * (g.th < 1.0 ? FxBlocks<true>::value : FxBlocks<false>::value);
    const long long cmax = (units + 3) / 4;
    if (c > cmax) c = cmax;
    if (c < 1) c = 1;
    gx = (int)c;
    gy = gz = 1;
    chunk = (int)((units + c - 1) / c);
    return gx;
}

cudaError_t launch_residual_fx(const GeoFX& f, const Geo& g, const double* U, const double* u0, const double* gdt,
                               const float* igamf, float* s, double* r_out, double* partials, const Ctl* ctl,
                               cudaStream_t st, int rout_mode) {
    int gx, gy, gz, chunk;
    residual_fx_grid(g, gx, gy, gz, chunk);
    const dim3 grid(gx), blk(kFxThreads);
#define PINT_RFX(D, H, R, C) \
    return launch_pdl(k_residual_fx<D, H, R, C>, grid, blk, 0, st, f, U, u0, gdt, igamf, s, r_out, partials, ctl)
    const bool rout = rout_mode != 0;
    if (f.cube) {
        if (g.dim == 2) { if (rout) PINT_RFX(2, false, true, true); else PINT_RFX(2, false, false, true); }
        else { if (rout) PINT_RFX(1, false, true, true); else PINT_RFX(1, false, false, true); }
    }
    if (g.dim == 2) {
        if (rout) { if (f.half) PINT_RFX(2, true, true, false); else PINT_RFX(2, false, true, false); }
        else { if (f.half) PINT_RFX(2, true, false, false); else PINT_RFX(2, false, false, false); }
    } else {
        if (rout) { if (f.half) PINT_RFX(1, true, true, false); else PINT_RFX(1, false, true, false); }
        else { if (f.half) PINT_RFX(1, true, false, false); else PINT_RFX(1, false, false, false); }
    }
#undef PINT_RFX
}

}  // namespace pint
