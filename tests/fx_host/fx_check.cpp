// Host-side checks of the block fixed-point helpers (fx.cuh) against exact
// 128-bit integer and long double arithmetic on seeded random arguments.
// Prints one line per helper: "<name> <checked> <failures> <worst>".
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <random>

#include "fx.cuh"

using namespace pint;

static double bits_to_double(uint64_t b) {
    double d;
    memcpy(&d, &b, 8);
    return d;
}

int main(int argc, char** argv) {
    const long n = argc > 1 ? atol(argv[1]) : 200000;
    std::mt19937_64 rng(20230427);

    // fx_from_f64_fast: trunc(|u| 2^(56-E)) with the sign of u, E >= the tile's exponent
    {
        long bad = 0;
        for (long i = 0; i < n; ++i) {
            const int ex = 1 + (int)(rng() % 2046);                   // normal doubles
            const uint64_t b = (rng() & 0x800FFFFFFFFFFFFFull) | ((uint64_t)ex << 52);
            const double u = bits_to_double(b);
            int E = ex - 1022 + (int)(rng() % 70);                    // |u| < 2^E
            if (E < -958) E = -958;
            if (ex - 1022 > E) continue;
            const int64_t got = fx_from_f64_fast((uint32_t)(b >> 32), (uint32_t)b, E);
            // exact: |u| = m 2^(ex-1075), in units 2^(E-56): m 2^(ex-1019-E)
            const __int128 m = (__int128)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
            const int sh = ex - 1019 - E;
            __int128 v = sh >= 0 ? (m << sh) : (sh <= -127 ? 0 : (m >> -sh));
            if (u < 0) v = -v;
            if ((__int128)got != v) ++bad;
        }
        printf("from_f64 %ld %ld 0\n", n, bad);
    }
    // fx_mul_shr: floor(L M / 2^S) for the sizes the residual uses
    {
        long bad = 0;
        for (long i = 0; i < n; ++i) {
            const int bl = 1 + (int)(rng() % 62), bm = 1 + (int)(rng() % 53);
            int64_t L = (int64_t)(rng() >> (64 - bl));
            if (rng() & 1) L = -L;
            const int64_t M = (int64_t)(rng() >> (64 - bm));
            const int S = (int)(rng() % 136);
            const __int128 p = (__int128)L * M;
            if (S < 127 && ((p >> S) > (__int128)INT64_MAX || (p >> S) < (__int128)INT64_MIN)) continue;
            const __int128 want = S >= 127 ? (p < 0 ? -1 : 0) : (p >> S);
            if ((__int128)fx_mul_shr(L, M, S) != want) ++bad;
        }
        printf("mul_shr %ld %ld 0\n", n, bad);
    }
    // fx_split_f64 + fx_to_f32_pair: R g 2^k within 7 2^-25 relative
    {
        long bad = 0;
        long double worst = 0;
        for (long i = 0; i < n; ++i) {
            const int ex = 900 + (int)(rng() % 250);
            const uint64_t gb = (rng() & 0x000FFFFFFFFFFFFFull) | ((uint64_t)ex << 52);
            float Gh, Gl;
            int e;
            fx_split_f64(gb, Gh, Gl, e);
            const long double g = (long double)bits_to_double(gb);
            const long double gpair = ((long double)Gh + (long double)Gl) * ldexpl(1.0L, e - 1046);
            if (fabsl(gpair - g) > ldexpl(g, -48)) ++bad;
            const int br = (int)(rng() % 63);
            int64_t R = (int64_t)(rng() >> (63 - br)) >> 1;
            if (rng() & 1) R = -R;
            // pick X so that the result is near 1 in magnitude, in the normal range
            const int X = -(br + (e - 1046) + 23) + (int)(rng() % 40) - 20;
            const int k = X + e - 1046;
            float f1, f2;
            {
                int k1 = k >> 1, k2 = k - k1;
                uint32_t b1 = (uint32_t)(k1 + 127) << 23, b2 = (uint32_t)(k2 + 127) << 23;
                memcpy(&f1, &b1, 4);
                memcpy(&f2, &b2, 4);
            }
            const float got = fx_to_f32_pair(R, Gh, Gl, f1, f2);
            const long double exact = (long double)R * g * ldexpl(1.0L, X);
            if (R == 0) {
                if (got != 0.0f) ++bad;
                continue;
            }
            const long double rel = fabsl(((long double)got - exact) / exact);
            if (rel > worst) worst = rel;
            if (rel > 7.0L * ldexpl(1.0L, -25)) ++bad;
        }
        printf("to_f32_pair %ld %ld %.3Le\n", n, bad, worst);
    }
    return 0;
}
