// k_jacobian.cu - the space-varying averaged Jacobian of Eq. 4.12 (paper-
// literal PinT-I / PinT-II): its field J~(x) = mean over the time levels of
// 3 u_n(x)^2, the variable-coefficient spatial operator of Step 2 applied to
// every frequency slice of the spectrum,
//   M_k y = lambda_1k y + lambda_2k (c2 Lap^2 y + Lap((c1 - J~) y)) + lambda_3k Lap y,
// (PinT-I: c1 = 1, lambda_3k = 0; PinT-II: c1 = 0, lambda_3k = 1 - dt lambda_1k),
// and the kernels of the inner flexible GMRES that solves it: complex vector
// kernels and the small one-CTA steps that keep its Hessenberg matrix, Givens
// rotations and stop test on the device.
#include "ff.cuh"
#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

// jt[p] = 3/nt sum_n u_n[p]^2 from the FP64 iterate (uff == nullptr) or the float-float one.
template <class T>
__global__ void k_jtilde(const double* __restrict__ U, const float2* __restrict__ uff, int nt, int nspace,
                         T* __restrict__ jt) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nspace; p += gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int n = 0; n < nt; ++n) {
            const double u = uff ? (double)uff[(size_t)n * nspace + p].x : U[(size_t)n * nspace + p];
            a = fma(u, u, a);
        }
        jt[p] = (T)(3.0 * a / nt);
    }
}

// Reflected index of a halo point (same boundary treatment as the residual):
// returns -1 for a zero ghost (simply supported), sets the sign.
__device__ __forceinline__ int refl_index(int g, int n, int bc, float& sgn) {
    if (bc == 1) return g < 0 ? -1 - g : (g >= n ? 2 * n - 1 - g : g);
    if (bc == 2) return g < 0 ? -g : (g >= n ? 2 * (n - 1) - g : g);
    if (g == -1 || g == n) return -1;
    if (g < -1) { sgn = -sgn; return -2 - g; }
    if (g > n) { sgn = -sgn; return 2 * n - g; }
    return g;
}

// One CTA: a 32 x 8 tile of one frequency slice k = blockIdx.z (1-D: 256 x 1).
template <class T, int DIM>
__global__ void __launch_bounds__(256) k_apply_M(Geo g, int nk, const c_t<T>* __restrict__ Y, c_t<T>* __restrict__ W,
                                                 const T* __restrict__ jt, Tabs<T> tb, T c2, T c1,
                                                 const int* __restrict__ skip, const c_t<T>* __restrict__ B) {
    using C = c_t<T>;
    if (skip && *skip) return;
    constexpr int TX = DIM == 2 ? 32 : 256, TY = DIM == 2 ? 8 : 1, HY = DIM == 2 ? 2 : 0;
    constexpr int SX = TX + 4, SY = TY + 2 * HY, LX = TX + 2, LY = TY + (DIM == 2 ? 2 : 0);
    __shared__ C sy[SY * SX];   // y
    __shared__ C sq[SY * SX];   // (c1 - J~) y
    __shared__ C sL[LY * LX];   // Lap y
    const int k = blockIdx.z;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const C* Yk = Y + (size_t)k * g.nspace;
    for (int e = threadIdx.x; e < SX * SY; e += TX * TY) {
        const int ix = e % SX, iy = e / SX;
        float sgn = 1.f;
        const int gx = refl_index(x0 - 2 + ix, g.nx, g.bc, sgn);
        const int gy = DIM == 2 ? refl_index(y0 - HY + iy, g.ny, g.bc, sgn) : 0;
        C v = mkc(T(0), T(0));
        T q = T(0);
        if (gx >= 0 && gx < g.nx && gy >= 0 && (DIM == 1 || gy < g.ny)) {
            const int idx = (DIM == 2 ? gy * g.nx : 0) + gx;
            v = scalec(Yk[idx], T(sgn));
            q = c1 - jt[idx];
        }
        sy[e] = v;
        sq[e] = scalec(v, q);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LX * LY; e += TX * TY) {
        const int ix = e % LX, iy = e / LX;
        const int c = (DIM == 2 ? (iy + 1) * SX : 0) + ix + 1;
        C v = scalec(sy[c - 1] + sy[c + 1] - scalec(sy[c], T(2)), T(g.ihx2));
        if (DIM == 2) v = v + scalec(sy[c - SX] + sy[c + SX] - scalec(sy[c], T(2)), T(g.ihy2));
        sL[e] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= g.nx || (DIM == 2 && gy >= g.ny)) return;
    const int cl = (DIM == 2 ? (ty + 1) * LX : 0) + tx + 1;
    const int cu = (ty + HY) * SX + tx + 2;
    const C L = sL[cl];
    C L2 = scalec(sL[cl - 1] + sL[cl + 1] - scalec(L, T(2)), T(g.ihx2));
    if (DIM == 2) L2 = L2 + scalec(sL[cl - LX] + sL[cl + LX] - scalec(L, T(2)), T(g.ihy2));
    C Lq = scalec(sq[cu - 1] + sq[cu + 1] - scalec(sq[cu], T(2)), T(g.ihx2));
    if (DIM == 2) Lq = Lq + scalec(sq[cu - SX] + sq[cu + SX] - scalec(sq[cu], T(2)), T(g.ihy2));
    const C op = scalec(L2, c2) + Lq;                       // c2 Lap^2 y + Lap((c1 - J~) y)
    const C l1 = tb.lam1[k], l2 = tb.lam2[k];
    C w = cmul(l1, sy[cu]) + cmul(l2, op);
    if (tb.dte != T(0)) w = w + cmul(mkc(T(1) - tb.dte * l1.x, -tb.dte * l1.y), L);   // lambda_3k Lap y
    const size_t o = (size_t)k * g.nspace + (DIM == 2 ? gy * g.nx : 0) + gx;
    W[o] = B ? B[o] - w : w;
}

constexpr int kCDotThreads = 256;
constexpr int kGroup = 4;   // vectors handled per launch (register accumulators)

// The vectors of the inner solve hold nk frequency slices of ns points each.  The
// GMRES cycle runs on every slice separately (M is block-diagonal over the
// frequencies, so each block gets its own Krylov coefficients): the vector
// kernels below use a 2-D grid, blockIdx.y = slice k, blockIdx.x = one of nbx
// CTAs over that slice's points, and read slice k's coefficients.

// partials[((k nbx + bx) ldp + i0 + i) 2 + {0,1}] = that CTA's part of <v_i, w>_k = sum conj(v_i) w, i < G.
template <class T, int G>
__global__ void __launch_bounds__(kCDotThreads) k_cmulti_dot(const c_t<T>* __restrict__ w, const c_t<T>* __restrict__ V,
                                                            size_t ld, size_t ns, int ldp, int i0,
                                                            double* __restrict__ partials, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ double red[kCDotThreads / 32][G][2];
    const size_t base = (size_t)blockIdx.y * ns;
    // each thread accumulates its strided elements in the vectors' own precision
    // (complex64: FP32, a few hundred terms at most); the CTA sum is taken in FP64
    T re[G], im[G];
#pragma unroll
    for (int i = 0; i < G; ++i) re[i] = im[i] = T(0);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < ns; e += (size_t)gridDim.x * blockDim.x) {
        const c_t<T> we = w[base + e];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const c_t<T> v = V[i * ld + base + e];
            re[i] = fma(v.x, we.x, fma(v.y, we.y, re[i]));
            im[i] = fma(v.x, we.y, fma(-v.y, we.x, im[i]));
        }
    }
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int i = 0; i < G; ++i) {
        const double a = warp_sum((double)re[i]), b = warp_sum((double)im[i]);
        if (lane == 0) { red[warp][i][0] = a; red[warp][i][1] = b; }
    }
    __syncthreads();
    if (threadIdx.x < G) {
        const int i = threadIdx.x;
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kCDotThreads / 32; ++q) { a += red[q][i][0]; b += red[q][i][1]; }
        const size_t cta = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        partials[(cta * ldp + i0 + i) * 2] = a;
        partials[(cta * ldp + i0 + i) * 2 + 1] = b;
    }
}

// out = (w + sum_i c_{k,i} v_i) * post_k on slice k, i < G (i0 + i < nlim, and
// < *nlimd when given: the vectors beyond are not read), with c_k from slice k's
// state (set sel) and post_k its scale (when post is set); out = w when null.
// Arithmetic in the vectors' precision.
template <class T, int G>
__global__ void k_cmulti_axpy(c_t<T>* __restrict__ w, const c_t<T>* __restrict__ V, size_t ld, size_t ns,
                              const GmK* __restrict__ gk, int sel, const int* __restrict__ skip, int nlim,
                              const int* __restrict__ nlimd, int i0, c_t<T>* __restrict__ out, int post) {
    if (skip && *skip) return;
    const GmK& s = gk[blockIdx.y];
    if (nlimd) nlim = min(nlim, *nlimd);
    const int ng = max(0, min(G, nlim - i0));
    const T ps = post ? (T)s.scale : T(1);
    if (!out) out = w;
    if (ng <= 0 && out == w && !post) return;
    const double2* c = sel == GM_COEF ? s.coef : (sel == GM_COEFA ? s.coefA : s.y);
    T cr[G], ci[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
        cr[i] = i < ng ? (T)c[i0 + i].x : T(0);
        ci[i] = i < ng ? (T)c[i0 + i].y : T(0);
    }
    const size_t base = (size_t)blockIdx.y * ns;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < ns; e += (size_t)gridDim.x * blockDim.x) {
        T xr = w[base + e].x, xi = w[base + e].y;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            if (i >= ng) break;
            const c_t<T> v = V[i * ld + base + e];
            xr = fma(cr[i], v.x, fma(-ci[i], v.y, xr));
            xi = fma(cr[i], v.y, fma(ci[i], v.x, xi));
        }
        out[base + e] = mkc(xr * ps, xi * ps);
    }
}

// z = a x + b y (real scalars; y may be nullptr; a = *sdev when sdev is given)
template <class T>
__global__ void k_caxpby(c_t<T>* __restrict__ z, T a, const c_t<T>* __restrict__ x, T b, const c_t<T>* __restrict__ y,
                         size_t n, const int* __restrict__ skip, const double* __restrict__ sdev) {
    if (skip && *skip) return;
    if (sdev) a = (T)*sdev;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        c_t<T> v = scalec(x[e], a);
        if (y) v = v + scalec(y[e], b);
        z[e] = v;
    }
}

// ---------------------------------------------------------------------------
// Scalar steps of the inner flexible GMRES: one CTA per frequency slice.
// ---------------------------------------------------------------------------
constexpr int kGmThreads = 128;

__device__ __forceinline__ double2 gm_mul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 gm_conj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 gm_scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 gm_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 gm_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double gm_abs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double gm_norm(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 gm_div(double2 a, double2 b) {
    const double d = gm_norm(b);
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// out[i] = sum over the slice's nbx CTAs, in CTA order, of the partials of
// vector i < nv: warp w adds the values v = w, w + 4, ... (re and im of each
// vector), each lane a fixed strided subset, then a fixed shuffle tree.
__device__ void gm_reduce(const double* __restrict__ part, int nbx, int nv, double2* out) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const double* pk = part + (size_t)blockIdx.x * nbx * nv * 2;
    double* o = reinterpret_cast<double*>(out);
    for (int v = warp; v < 2 * nv; v += kGmThreads / 32) {
        double a = 0.0;
        for (int q = lane; q < nbx; q += 32) a += pk[((size_t)q * nv + v / 2) * 2 + (v & 1)];
        a = warp_sum(a);
        if (lane == 0) o[v] = a;
    }
    __syncthreads();
}

// Start of a cycle: every slice running, no second Gram-Schmidt pass requested.
__global__ void k_gm_reset(GmHead* h) {
    for (int i = threadIdx.x; i < kMaxKrylov; i += blockDim.x) h->skip_re[i] = 1;
    if (threadIdx.x == 0) {
        h->ndone = 0;
        h->skip = 0;
        h->jmax = 0;
        h->ictl.status = ST_RUNNING;
    }
}

// A slice leaves the cycle: its coefficients and scale become 0 (its basis vectors
// are then zero and stay finite), and the last slice to leave stops the cycle.
__device__ void gm_leave(GmK& s, GmHead* h, int nk) {
    s.done = 1;
    s.scale = 0.0;
    if (atomicAdd(&h->ndone, 1) + 1 == nk) {
        h->skip = 1;
        h->ictl.status = 0;
    }
}

__global__ void __launch_bounds__(kGmThreads) k_gm_init(const double* __restrict__ part_bb,
                                                        const double* __restrict__ part_rr, int nbx,
                                                        const Ctl* __restrict__ octl, GmHead* h, GmK* gk, int nk,
                                                        double tol) {
    __shared__ double2 bb[1], rr[1];
    gm_reduce(part_bb, nbx, 1, bb);
    gm_reduce(part_rr, nbx, 1, rr);
    if (threadIdx.x != 0) return;
    GmK& s = gk[blockIdx.x];
    const double bn = sqrt(fmax(bb[0].x, 0.0)), beta = sqrt(fmax(rr[0].x, 0.0));
    if (blockIdx.x == 0) h->ictl.jbar = octl->jbar;
    s.done = 0;
    s.j = 0;
    s.bn = bn;
    s.scale = beta > 0.0 ? 1.0 / beta : 0.0;
    s.gv[0] = make_double2(beta, 0.0);
    // a slice already solved (or zero), or every slice when the outer iteration has stopped
    if (octl->status != ST_RUNNING || !(beta > tol * bn)) gm_leave(s, h, nk);
}

__global__ void __launch_bounds__(kGmThreads) k_gm_orth1(const double* __restrict__ part, int nbx, int j, GmHead* h,
                                                         GmK* gk) {
    GmK& s = gk[blockIdx.x];
    if (h->skip || s.done) {
        if (threadIdx.x == 0)
            for (int i = 0; i <= j; ++i) s.coef[i] = s.coefA[i] = make_double2(0.0, 0.0);
        return;
    }
    gm_reduce(part, nbx, j + 2, s.tmp);
    if (threadIdx.x != 0) return;
    const double ww = s.tmp[j + 1].x;
    double hh = 0.0;
    for (int i = 0; i <= j; ++i) {
        s.hcol[i] = s.tmp[i];
        hh += gm_norm(s.tmp[i]);
        s.coef[i] = gm_scale(s.tmp[i], -1.0);
    }
    const double hn2 = ww - hh;
    // ||w - sum h_i v_i||^2 = <w, w> - sum |h_i|^2 cancels: project once more
    s.reorth = hn2 > 1e-4 * ww ? 0 : 1;
    for (int i = 0; i <= j; ++i) s.coefA[i] = s.reorth ? s.coef[i] : make_double2(0.0, 0.0);
    if (s.reorth) h->skip_re[j] = 0;   // step j's second pass runs (for the slices that asked)
    s.hn2 = hn2;
}

__global__ void __launch_bounds__(kGmThreads) k_gm_orth2(const double* __restrict__ part, int nbx, int j, GmHead* h,
                                                         GmK* gk, int nk, double tol) {
    GmK& s = gk[blockIdx.x];
    // a slice that left earlier (its own flag), or all of them (the cycle stopped before this launch)
    const bool run = !s.done && !h->skip;
    if (run && s.reorth) gm_reduce(part, nbx, j + 2, s.tmp);   // the second pass ran: skip_re[j] was cleared
    if (threadIdx.x != 0 || !run) return;
    double hn2 = s.hn2;
    if (s.reorth) {
        double hh = 0.0;
        for (int i = 0; i <= j; ++i) {
            s.hcol[i] = gm_add(s.hcol[i], s.tmp[i]);
            hh += gm_norm(s.tmp[i]);
            s.coef[i] = gm_scale(s.tmp[i], -1.0);
        }
        hn2 = s.tmp[j + 1].x - hh;
    }
    const double hn = sqrt(fmax(hn2, 0.0));
    s.scale = hn > 0.0 ? 1.0 / hn : 0.0;
    double2* hc = s.hcol;
    hc[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {   // the previous rotations
        const double2 a = gm_add(gm_scale(hc[i], s.cs[i]), gm_mul(s.sn[i], hc[i + 1]));
        hc[i + 1] = gm_sub(gm_scale(hc[i + 1], s.cs[i]), gm_mul(gm_conj(s.sn[i]), hc[i]));
        hc[i] = a;
    }
    const double na = gm_abs(hc[j]), r = hypot(na, gm_abs(hc[j + 1]));
    if (r == 0.0) {
        s.cs[j] = 1.0;
        s.sn[j] = make_double2(0.0, 0.0);
    } else if (na == 0.0) {
        s.cs[j] = 0.0;
        s.sn[j] = gm_scale(gm_conj(hc[j + 1]), 1.0 / r);
    } else {
        s.cs[j] = na / r;
        s.sn[j] = gm_scale(gm_mul(gm_scale(hc[j], 1.0 / na), gm_conj(hc[j + 1])), 1.0 / r);
    }
    hc[j] = gm_add(gm_scale(hc[j], s.cs[j]), gm_mul(s.sn[j], hc[j + 1]));
    hc[j + 1] = make_double2(0.0, 0.0);
    s.gv[j + 1] = gm_scale(gm_mul(gm_conj(s.sn[j]), s.gv[j]), -1.0);
    s.gv[j] = gm_scale(s.gv[j], s.cs[j]);
    for (int i = 0; i <= j; ++i) s.H[i * kMaxKrylov + j] = hc[i];
    s.j = j + 1;
    h->jmax = j + 1;   // the same value from every slice still running
    if (gm_abs(s.gv[j + 1]) <= tol * s.bn || hn == 0.0) gm_leave(s, h, nk);
}

// y_k = H_k^{-1} g_k over slice k's completed steps (zero beyond them).
__global__ void k_gm_solve(GmK* gk) {
    if (threadIdx.x != 0) return;
    GmK& s = gk[blockIdx.x];
    const int j = s.j;
    for (int i = 0; i < kMaxKrylov; ++i) s.y[i] = make_double2(0.0, 0.0);
    for (int i = j - 1; i >= 0; --i) {
        double2 a = s.gv[i];
        for (int k = i + 1; k < j; ++k) a = gm_sub(a, gm_mul(s.H[i * kMaxKrylov + k], s.y[k]));
        s.y[i] = gm_div(a, s.H[i * kMaxKrylov + i]);
    }
}

static int grid_n(size_t n) {
    const size_t b = (n + 255) / 256;
    return (int)(b > 2 * 152 * 4 ? 2 * 152 * 4 : (b < 1 ? 1 : b));
}
// CTAs per slice of the per-slice vector kernels: about 2 x 152 x 4 in all.
int cdot_blocks(size_t ns, int nk) {
    const size_t per = (size_t)(2 * 152 * 4 + nk - 1) / nk;
    const size_t b = (ns + 255) / 256;
    return (int)(b < per ? (b < 1 ? 1 : b) : (per < 1 ? 1 : per));
}

template <class T>
void launch_jtilde(const double* U, const float2* uff, int nt, int nspace, T* jt, cudaStream_t st) {
    k_jtilde<T><<<grid_n(nspace), 256, 0, st>>>(U, uff, nt, nspace, jt);
}
template <class T>
void launch_apply_M(const Geo& g, int nk, const c_t<T>* Y, c_t<T>* W, const T* jt, const Tabs<T>& tb, double c2,
                    double c1, const int* skip, const c_t<T>* B, cudaStream_t st) {
    if (g.dim == 2) {
        dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, nk);
        k_apply_M<T, 2><<<grid, 256, 0, st>>>(g, nk, Y, W, jt, tb, (T)c2, (T)c1, skip, B);
    } else {
        dim3 grid((g.nx + 255) / 256, 1, nk);
        k_apply_M<T, 1><<<grid, 256, 0, st>>>(g, nk, Y, W, jt, tb, (T)c2, (T)c1, skip, B);
    }
}
// Groups of up to kGroup vectors per launch, register accumulators.
template <class T>
void launch_cmulti_dot(const c_t<T>* w, const c_t<T>* V, size_t ld, int nv, size_t ns, int nk, double* partials,
                       const int* skip, cudaStream_t st) {
    const dim3 grid(cdot_blocks(ns, nk), nk);
    for (int i0 = 0; i0 < nv; i0 += kGroup) {
        const c_t<T>* Vi = V + (size_t)i0 * ld;
        switch (nv - i0 >= kGroup ? kGroup : nv - i0) {
            case 1: k_cmulti_dot<T, 1><<<grid, kCDotThreads, 0, st>>>(w, Vi, ld, ns, nv, i0, partials, skip); break;
            case 2: k_cmulti_dot<T, 2><<<grid, kCDotThreads, 0, st>>>(w, Vi, ld, ns, nv, i0, partials, skip); break;
            case 3: k_cmulti_dot<T, 3><<<grid, kCDotThreads, 0, st>>>(w, Vi, ld, ns, nv, i0, partials, skip); break;
            default: k_cmulti_dot<T, 4><<<grid, kCDotThreads, 0, st>>>(w, Vi, ld, ns, nv, i0, partials, skip); break;
        }
    }
}
template <class T>
void launch_cmulti_axpy(c_t<T>* w, const c_t<T>* V, size_t ld, int nv, int nlim, size_t ns, int nk, const GmK* gk,
                        int sel, const int* skip, cudaStream_t st, c_t<T>* out, int post, const int* nlimd) {
    const dim3 grid(cdot_blocks(ns, nk), nk);
    if (nv == 0) {   // out = w * post only
        k_cmulti_axpy<T, 1><<<grid, 256, 0, st>>>(w, V, ld, ns, gk, sel, skip, 0, nullptr, 0, out, post);
        return;
    }
    for (int i0 = 0; i0 < nv; i0 += kGroup) {
        const c_t<T>* Vi = V + (size_t)i0 * ld;
        // the first group reads w and writes out; later groups update out in place; the last one scales
        c_t<T>* src = i0 == 0 ? w : (out ? out : w);
        const int ps = i0 + kGroup >= nv ? post : 0;
        switch (nv - i0 >= kGroup ? kGroup : nv - i0) {
            case 1: k_cmulti_axpy<T, 1><<<grid, 256, 0, st>>>(src, Vi, ld, ns, gk, sel, skip, nlim, nlimd, i0, out, ps); break;
            case 2: k_cmulti_axpy<T, 2><<<grid, 256, 0, st>>>(src, Vi, ld, ns, gk, sel, skip, nlim, nlimd, i0, out, ps); break;
            case 3: k_cmulti_axpy<T, 3><<<grid, 256, 0, st>>>(src, Vi, ld, ns, gk, sel, skip, nlim, nlimd, i0, out, ps); break;
            default: k_cmulti_axpy<T, 4><<<grid, 256, 0, st>>>(src, Vi, ld, ns, gk, sel, skip, nlim, nlimd, i0, out, ps); break;
        }
    }
}
template <class T>
void launch_caxpby(c_t<T>* z, double a, const c_t<T>* x, double b, const c_t<T>* y, size_t n, const int* skip,
                   const double* sdev, cudaStream_t st) {
    k_caxpby<T><<<grid_n(n), 256, 0, st>>>(z, (T)a, x, (T)b, y, n, skip, sdev);
}
void launch_gm_reset(GmHead* h, cudaStream_t st) { k_gm_reset<<<1, 32, 0, st>>>(h); }
void launch_gm_init(const double* part_bb, const double* part_rr, int nbx, const Ctl* octl, GmHead* h, GmK* gk,
                    int nk, double tol, cudaStream_t st) {
    k_gm_init<<<nk, kGmThreads, 0, st>>>(part_bb, part_rr, nbx, octl, h, gk, nk, tol);
}
void launch_gm_orth1(const double* part, int nbx, int j, GmHead* h, GmK* gk, int nk, cudaStream_t st) {
    k_gm_orth1<<<nk, kGmThreads, 0, st>>>(part, nbx, j, h, gk);
}
void launch_gm_orth2(const double* part, int nbx, int j, GmHead* h, GmK* gk, int nk, double tol, cudaStream_t st) {
    k_gm_orth2<<<nk, kGmThreads, 0, st>>>(part, nbx, j, h, gk, nk, tol);
}
void launch_gm_solve(GmK* gk, int nk, cudaStream_t st) { k_gm_solve<<<nk, 32, 0, st>>>(gk); }

#define PINT_INST(T)                                                                                              \
    template void launch_jtilde<T>(const double*, const float2*, int, int, T*, cudaStream_t);                      \
    template void launch_apply_M<T>(const Geo&, int, const c_t<T>*, c_t<T>*, const T*, const Tabs<T>&, double,    \
                                    double, const int*, const c_t<T>*, cudaStream_t);                             \
    template void launch_cmulti_dot<T>(const c_t<T>*, const c_t<T>*, size_t, int, size_t, int, double*,          \
                                       const int*, cudaStream_t);                                                 \
    template void launch_cmulti_axpy<T>(c_t<T>*, const c_t<T>*, size_t, int, int, size_t, int, const GmK*, int,   \
                                        const int*, cudaStream_t, c_t<T>*, int, const int*);                      \
    template void launch_caxpby<T>(c_t<T>*, double, const c_t<T>*, double, const c_t<T>*, size_t, const int*,      \
                                   const double*, cudaStream_t);
PINT_INST(float)
PINT_INST(double)
#undef PINT_INST

}  // namespace pint
