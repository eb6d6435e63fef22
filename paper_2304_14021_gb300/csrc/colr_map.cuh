// colr_map.cuh - integer maps of the Step 2 passes over columns in register
// four-step form (k_spatial.cu, k_cols_dct_fdi_r): the even/odd reordering of
// the DCT-II, the tile's 16-byte chunk layout, the lanes of a column and their
// DCT-pair partners, and the order in which the pair solve updates a lane's
// entries.  __host__ __device__ so that their properties (a bijective layout,
// conflict-free shared-memory accesses, an involutive partner map, every
// entry updated once with its partner p + q = 0 mod N) can be checked on the
// host.
#pragma once

#if defined(__CUDACC__)
#define CR_HD __host__ __device__ __forceinline__
#else
#define CR_HD inline
#endif

namespace pint {

// position of x_i in the even/odd reordered sequence v (v_j = x_2j, v_{n-1-j} = x_{2j+1})
CR_HD int dct_pos(int i, int n) { return (i & 1) ? n - 1 - (i >> 1) : (i >> 1); }

namespace colr {

// the tile holds 8 column pairs; pair pr, reordered row r is the 16-byte chunk
// pr*N + (r ^ ((r >> lg) & (G - 1)) ^ pr) with G = 2^lg = sqrt(N) lanes per
// column, column 2 pr + h at byte 8 h of it: the first DFT step's rows
// s + G j and the exchange's rows j + G s then land on G different chunk
// slots mod G
CR_HD int chunk(int n, int pr, int r) {
    const int lg = n == 64 ? 3 : 4;
    return pr * n + ((r ^ ((r >> lg) & ((1 << lg) - 1))) ^ pr);
}

// Lane layout of a CTA of 16 G threads: lane bits 0-2 are the low bits of s,
// bit 3 selects the column of the pair, bit 4 is the high bit of s (G = 16)
// or the pair within the warp (G = 8).  s is the lane's index within its
// column (j1 in the first DFT step, k2 in the second).
struct Lane {
    int s, half, cp, c, partner;
};
CR_HD Lane lane(int g, int tid) {
    const int ln = tid % 32, warp = tid / 32;
    Lane l;
    l.half = (ln >> 3) & 1;
    l.s = g == 16 ? (ln & 7) | ((ln >> 4) << 3) : (ln & 7);
    l.cp = g == 16 ? warp : 2 * warp + (ln >> 4);
    l.c = 2 * l.cp + l.half;
    const int sp = (g - l.s) % g;   // the partner holds entries N - p
    l.partner = g == 16 ? (sp & 7) | (l.half << 3) | ((sp >> 3) << 4) : sp | (ln & 24);
    return l;
}

// Step m of the pair solve (m = 0 .. G/2 - 1) updates entries a and b of lane
// s (entry k1 holds frequency p = s + G k1).  For s != 0 entry m pairs with
// the partner's entry G-1-m and vice versa; lane 0 pairs (k1, G - k1) within
// itself, so it takes entries m+1 and G-1-m and leaves entry 0 for the end.
constexpr int pair_b(int g, int m) { return g - 1 - m; }
constexpr int pair_a_lane0(int g, int m) { return (m + 1) % g; }
CR_HD int pair_a(int g, int s, int m) { return s == 0 ? pair_a_lane0(g, m) : m; }

}  // namespace colr
}  // namespace pint
