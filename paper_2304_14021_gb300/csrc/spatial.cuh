// spatial.cuh - shared pieces of the Step 2 kernels (k_spatial.cu, k_dst.cu):
// the pass modes and the shifted eigenvalue denominator of Eq. 2.8 / Eq. 4.14.
#pragma once

#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

enum { MODE_FWD = 0, MODE_INV = 1, MODE_FDI = 2, MODE_PACK = 3 };

template <class T>
__device__ __forceinline__ c_t<T> shift_den(const Tabs<T>& tb, int k, T Lam, T c2, T c1) {
    const T mu = c2 * Lam * Lam + c1 * Lam;
    const c_t<T> l1 = tb.lam1[k], l2 = tb.lam2[k];
    c_t<T> d = mkc(l1.x + l2.x * mu, l1.y + l2.y * mu);
    if (tb.dte != T(0)) {   // PinT-II: + lambda_3k Lam, lambda_3k = alpha^{1/N_t} e^{-2 pi i k/N_t} = 1 - dt lambda_1k
        d.x += (T(1) - tb.dte * l1.x) * Lam;
        d.y -= tb.dte * l1.y * Lam;
    }
    return d;
}

template <class T>
__device__ __forceinline__ T solve_c1(SolveCoef co, const Ctl* ctl) {
    return co.ch ? T(co.c1 - ctl->jbar) : T(co.c1);
}

}  // namespace pint
