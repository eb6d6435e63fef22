// Host checks of the integer maps of the register four-step column pass
// (colr_map.cuh).  Prints one line per property: "<name> <checked> <failures>".
#include <stdio.h>

#include <set>
#include <vector>

#include "colr_map.cuh"

using namespace pint;

static void report(const char* name, long checked, long bad) { printf("%s %ld %ld\n", name, checked, bad); }

int main() {
    const int sizes[2] = {64, 256};
    // dct_pos is a permutation of 0..n-1 with x_2j at j and x_2j+1 at n-1-j
    {
        long checked = 0, bad = 0;
        for (int n : sizes) {
            std::vector<int> seen(n, 0);
            for (int i = 0; i < n; ++i) {
                const int p = dct_pos(i, n);
                ++checked;
                if (p < 0 || p >= n || seen[p]++) ++bad;
                if ((i % 2 == 0 && p != i / 2) || (i % 2 == 1 && p != n - 1 - i / 2)) ++bad;
            }
        }
        report("dct_pos", checked, bad);
    }
    // the chunk layout is a bijection of (pair, row) onto the tile's 8 N chunks
    {
        long checked = 0, bad = 0;
        for (int n : sizes) {
            std::vector<int> seen(8 * n, 0);
            for (int pr = 0; pr < 8; ++pr)
                for (int r = 0; r < n; ++r) {
                    const int c = colr::chunk(n, pr, r);
                    ++checked;
                    if (c < 0 || c >= 8 * n || seen[c]++) ++bad;
                }
        }
        report("chunk_bijection", checked, bad);
    }
    // copies in and out: 16-byte accesses, thread (pair tid % 8, row tid / 8 + ...):
    // every 8 consecutive lanes (one 128-byte phase) hit 8 different 16-byte bank groups
    {
        long checked = 0, bad = 0;
        for (int n : sizes) {
            const int nth = n == 64 ? 128 : 256, rstep = nth / 8;
            for (int i = 0; i < n / rstep; ++i)
                for (int q0 = 0; q0 < nth; q0 += 8) {
                    std::set<int> groups;
                    for (int t = q0; t < q0 + 8; ++t) {
                        const int y = t / 8 + rstep * i;
                        groups.insert(colr::chunk(n, t % 8, dct_pos(y, n)) % 8);
                    }
                    ++checked;
                    if ((int)groups.size() != 8) ++bad;
                }
        }
        report("copy_banks", checked, bad);
    }
    // lanes: each (column, s) once per CTA, the partner an involution in the same
    // warp and column with s' = (G - s) mod G
    {
        long checked = 0, bad = 0;
        for (int n : sizes) {
            const int g = n == 64 ? 8 : 16, nth = 16 * g;
            std::set<int> seen;
            for (int t = 0; t < nth; ++t) {
                const colr::Lane l = colr::lane(g, t);
                ++checked;
                if (l.c < 0 || l.c >= 16 || l.s < 0 || l.s >= g || !seen.insert(l.c * g + l.s).second) ++bad;
                const int pt = (t / 32) * 32 + l.partner;
                const colr::Lane m = colr::lane(g, pt);
                if (l.partner < 0 || l.partner >= 32 || m.c != l.c || m.s != (g - l.s) % g) ++bad;
                if (colr::lane(g, (pt / 32) * 32 + m.partner).s != l.s || (pt / 32) * 32 + m.partner != t) ++bad;
            }
        }
        report("lanes_partner", checked, bad);
    }
    // shared-memory accesses of the two DFT steps (8 bytes per lane): in each half-warp
    // the 16 lanes hit 16 different 8-byte bank pairs, for the reads of rows s + G j and
    // the exchange writes of rows j + G s
    {
        long checked = 0, bad = 0;
        for (int n : sizes) {
            const int g = n == 64 ? 8 : 16, nth = 16 * g;
            for (int pattern = 0; pattern < 2; ++pattern)
                for (int j = 0; j < g; ++j)
                    for (int h0 = 0; h0 < nth; h0 += 16) {
                        std::set<int> pairs;
                        for (int t = h0; t < h0 + 16; ++t) {
                            const colr::Lane l = colr::lane(g, t);
                            const int r = pattern == 0 ? l.s + g * j : j + g * l.s;
                            const long byte = 16L * colr::chunk(n, l.cp, r) + 8 * l.half;
                            pairs.insert((int)((byte / 8) % 16));
                        }
                        ++checked;
                        if ((int)pairs.size() != 16) ++bad;
                    }
        }
        report("dft_banks", checked, bad);
    }
    // the pair solve: over steps m = 0 .. G/2 - 1 (and entry 0 of lane 0 at the end)
    // every entry of every lane is updated once, and the value taken for it is its
    // pair's: p + q = 0 mod N with p = s + G k1
    {
        long checked = 0, bad = 0;
        for (int n : sizes) {
            const int g = n == 64 ? 8 : 16;
            for (int s = 0; s < g; ++s) {
                std::vector<int> count(g, 0);
                const int sp = (g - s) % g;
                for (int m = 0; m < g / 2; ++m) {
                    const int a = colr::pair_a(g, s, m), b = colr::pair_b(g, m);
                    count[a]++;
                    if (b != a) count[b]++;
                    // pair of a: lane 0 its own entry b; else the partner's entry b
                    // pair of b: lane 0 its own entry a; else the partner's entry m (its a)
                    const int qa = s == 0 ? s + g * b : sp + g * b;
                    const int qb = s == 0 ? s + g * a : sp + g * colr::pair_a(g, sp, m);
                    checked += 2;
                    if ((s + g * a + qa) % n != 0) ++bad;
                    if ((s + g * b + qb) % n != 0) ++bad;
                }
                if (s == 0) count[0]++;
                for (int k = 0; k < g; ++k) {
                    ++checked;
                    if (count[k] != 1) ++bad;
                }
            }
        }
        report("pair_schedule", checked, bad);
    }
    return 0;
}
