// k_residual.cu - FP64 all-at-once residual, its norm, and the per-iteration
// control reduction.
//
// Residual (Eq. 2.6 / Eq. 4.8 with alpha = 0) of the theta-method:
//   r_n = (u_{n-1} - u_n)/dt - theta A(u_n) - (1 - theta) A(u_{n-1}),
//   u_{-1} := u0 (the initial condition),  A(u) = c2 Lap^2 u + c1 Lap u + cN Lap(u^3).
// With U = 0 the first level is the right-hand side b_1 = u0/dt - (1-theta) A(u0).
// Lap is the centred 3-point (1-D) / 5-point (2-D) difference of Eq. 2.4.  The
// boundary conditions enter as reflections of the grid function: even about
// the cell face for cell-centred Neumann (u_{-1} = u_0), even about the end
// vertex for vertex-centred Neumann (u_{-1} = u_1), odd about the
// boundary vertex for simply supported (u_{-1} = 0, u_{-2} = -u_0).  With
// those ghost values Lap u is then correct on the ghost layer as well
// (Neumann: Lap u mirrors; simply supported: Lap u = 0 on the boundary), so
// Lap^2 u = Lap(Lap u) needs no further boundary logic.
#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

// Reflected read of one time level (n fixed) at integer grid index (gx, gy).
__device__ __forceinline__ double ext_read(const double* __restrict__ u, int gx, int gy, int nx, int ny,
                                           int dim, int bc) {
    double sgn = 1.0;
    if (bc == 1) {  // Neumann, cell-centred: even about the faces at -1/2 and n-1/2
        if (gx < 0) gx = -1 - gx;
        else if (gx >= nx) gx = 2 * nx - 1 - gx;
        if (dim == 2) {
            if (gy < 0) gy = -1 - gy;
            else if (gy >= ny) gy = 2 * ny - 1 - gy;
        }
    } else if (bc == 2) {  // Neumann, vertex grid: even about the end vertices 0 and n-1
        if (gx < 0) gx = -gx;
        else if (gx >= nx) gx = 2 * (nx - 1) - gx;
        if (dim == 2) {
            if (gy < 0) gy = -gy;
            else if (gy >= ny) gy = 2 * (ny - 1) - gy;
        }
    } else {  // simply supported, vertex grid: odd about the boundary vertices -1 and n
        if (gx == -1 || gx == nx) return 0.0;
        if (gx < -1) { gx = -2 - gx; sgn = -sgn; }
        else if (gx > nx) { gx = 2 * nx - gx; sgn = -sgn; }
        if (dim == 2) {
            if (gy == -1 || gy == ny) return 0.0;
            if (gy < -1) { gy = -2 - gy; sgn = -sgn; }
            else if (gy > ny) { gy = 2 * ny - gy; sgn = -sgn; }
        }
    }
    if (gx < 0 || gx >= nx || (dim == 2 && (gy < 0 || gy >= ny))) return 0.0;  // tiles wider than the grid
    return sgn * u[(dim == 2 ? gy * nx : 0) + gx];
}

template <int DIM> struct ResTile;
template <> struct ResTile<1> { static constexpr int TX = 256, TY = 1; };
template <> struct ResTile<2> { static constexpr int TX = 32, TY = 8; };

// One CTA: spatial tile TX x TY, time levels [n0, n0 + chunk).
// Outputs (each optional): r (FP64), s = gamma_n r_n cast to TS.
// partials[cta] = (sum r^2, sum u^2) over its points.
template <int DIM, class TS>
__global__ void __launch_bounds__(256) k_residual(Geo g, const double* __restrict__ U,
                                                  const double* __restrict__ u0,
                                                  const double* __restrict__ gam, double* __restrict__ r_out,
                                                  TS* __restrict__ s_out, double* __restrict__ partials,
                                                  const Ctl* __restrict__ ctl, int chunk) {
    if (ctl && ctl->status != ST_RUNNING) return;
    constexpr int TX = ResTile<DIM>::TX, TY = ResTile<DIM>::TY;
    constexpr int HY = DIM == 2 ? 2 : 0;
    constexpr int SX = TX + 4, SY = TY + 2 * HY;
    constexpr int LX = TX + 2, LY = TY + (DIM == 2 ? 2 : 0);
    __shared__ double su[SY * SX];
    __shared__ double sL[LY * LX];
    __shared__ double red[2][8];

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool inside = gx < g.nx && (DIM == 1 || gy < g.ny);
    const int pidx = (DIM == 2 ? gy * g.nx : 0) + gx;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(g.nt, n0 + chunk);
    // theta < 1 needs A(u_{n-1}); Eyre's splitting needs Lap u_{n-1}: both from one extra level before the chunk
    const bool prev = g.th < 1.0 || g.expl;

    double uprev = 0.0, Aprev = 0.0, Lprev = 0.0;
    if (inside) uprev = n0 == 0 ? u0[pidx] : (U ? U[(size_t)(n0 - 1) * g.nspace + pidx] : 0.0);
    double acc_r2 = 0.0, acc_u2 = 0.0;

    for (int n = prev ? n0 - 1 : n0; n < n1; ++n) {
        // level n (n = -1: u0; U == nullptr: the zero iterate)
        const double* un = n < 0 ? u0 : (U ? U + (size_t)n * g.nspace : nullptr);
        for (int e = threadIdx.x; e < SX * SY; e += TX * TY) {
            int ix = e % SX, iy = e / SX;
            su[e] = un ? ext_read(un, x0 - 2 + ix, y0 - HY + iy, g.nx, g.ny, DIM, g.bc) : 0.0;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < LX * LY; e += TX * TY) {
            int ix = e % LX, iy = e / LX;
            const int c = (DIM == 2 ? (iy + 1) * SX : 0) + ix + 1;  // su index of this L point
            double v = (su[c - 1] + su[c + 1] - 2.0 * su[c]) * g.ihx2;
            if (DIM == 2) v += (su[c - SX] + su[c + SX] - 2.0 * su[c]) * g.ihy2;
            sL[e] = v;
        }
        __syncthreads();
        if (inside) {
            const int cl = (DIM == 2 ? (ty + 1) * LX : 0) + tx + 1;
            const int cu = (ty + HY) * SX + tx + 2;
            const double L = sL[cl];
            double L2 = (sL[cl - 1] + sL[cl + 1] - 2.0 * L) * g.ihx2;
            if (DIM == 2) L2 += (sL[cl - LX] + sL[cl + LX] - 2.0 * L) * g.ihy2;
            const double u = su[cu];
            double A = g.c2 * L2 + (g.expl ? 0.0 : g.c1 * L);
            if (g.cN != 0.0) {
                double w0 = u * u * u;
                double we = su[cu + 1] * su[cu + 1] * su[cu + 1];
                double ww = su[cu - 1] * su[cu - 1] * su[cu - 1];
                double lw = (we + ww - 2.0 * w0) * g.ihx2;
                if (DIM == 2) {
                    double wn = su[cu - SX] * su[cu - SX] * su[cu - SX];
                    double ws = su[cu + SX] * su[cu + SX] * su[cu + SX];
                    lw += (wn + ws - 2.0 * w0) * g.ihy2;
                }
                A = fma(g.cN, lw, A);
            }
            if (n >= n0) {
                const double r = g.expl ? (uprev - u) * g.inv_dt - A - g.c1 * Lprev
                                 : prev ? (uprev - u) * g.inv_dt - g.th * A - (1.0 - g.th) * Aprev
                                        : (uprev - u) * g.inv_dt - A;
                const size_t o = (size_t)n * g.nspace + pidx;
                if (r_out) r_out[o] = r;
                if (s_out) s_out[o] = (TS)(gam[n] * r);
                acc_r2 = fma(r, r, acc_r2);
                acc_u2 = fma(u, u, acc_u2);
                uprev = u;
            }
            Aprev = A;
            Lprev = L;
        }
        __syncthreads();
    }
    // deterministic block reduction
    acc_r2 = warp_sum(acc_r2);
    acc_u2 = warp_sum(acc_u2);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) { red[0][warp] = acc_r2; red[1][warp] = acc_u2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (TX * TY) / 32; ++w) { a += red[0][w]; b += red[1][w]; }
        size_t cta = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[2 * cta] = a;
        partials[2 * cta + 1] = b;
    }
}

// partials[cta] = (sum u0^2, 0) over a 1-D chunking of u0.
__global__ void __launch_bounds__(256) k_norm2(const double* __restrict__ v, int n, double* __restrict__ partials) {
    __shared__ double red[8];
    double a = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a = fma(v[i], v[i], a);
    a = warp_sum(a);
    if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        partials[2 * blockIdx.x] = s;
        partials[2 * blockIdx.x + 1] = 0.0;
    }
}

// Sum the (a, b) partial pairs in a fixed order; one CTA of 256 threads.
__device__ void reduce_pairs(const double* __restrict__ partials, int np, double& A, double& B) {
    __shared__ double ra[8], rb[8];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) { a += partials[2 * i]; b += partials[2 * i + 1]; }
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x % 32 == 0) { ra[threadIdx.x / 32] = a; rb[threadIdx.x / 32] = b; }
    __syncthreads();
    A = 0.0;
    B = 0.0;
    for (int w = 0; w < 8; ++w) { A += ra[w]; B += rb[w]; }
}

// Start of a window: ||b|| = sqrt(sum of the partials) * scale (theta = 1:
// the partials of ||u0||^2 and scale 1/dt; theta < 1: those of ||b_1||^2 and
// scale 1), reset the iteration state.
__global__ void __launch_bounds__(256) k_begin_window(const double* __restrict__ partials, int np, double scale,
                                                      int max_iter, double tol, double tol_update, Ctl* ctl) {
    double A, B;
    reduce_pairs(partials, np, A, B);
    if (threadIdx.x == 0) {
        ctl->bnorm = sqrt(A) * scale;
        ctl->status = ST_RUNNING;
        ctl->iter = 0;
        ctl->max_iter = max_iter;
        ctl->tol = tol;
        ctl->tol_update = tol_update;
        ctl->dnorm = 1.0;
        ctl->rho0 = 0.0;
        ctl->rho = 0.0;
    }
}

// After the residual of iterate k: rho_k, jbar, stopping decision.  When the
// iteration runs as a CUDA-graph while-loop, this kernel also sets the loop
// condition (1 = run another iteration); it does so on every path, so a loop
// whose status is already final stops after this iteration.
__global__ void __launch_bounds__(256) k_after_residual(const double* __restrict__ partials, int np,
                                                        double inv_dof, Ctl* ctl, cudaGraphConditionalHandle cond,
                                                        int use_cond, const double* __restrict__ dpart, int ndp) {
    pdl_wait();
    if (ctl->status != ST_RUNNING) {
        if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    // Thread 0 loads the control fields of the decision first, so that their
    // latency overlaps the partial-sum loads instead of trailing the stores.
    int k = 0, max_iter = 0;
    double bn = 0.0, tol = 0.0, tol_upd = 0.0, rho0 = 0.0, h1 = 0.0, h2 = 0.0, h3 = 0.0, dh3 = 0.0;
    if (threadIdx.x == 0) {
        k = ctl->iter;
        max_iter = ctl->max_iter;
        bn = ctl->bnorm;
        tol = ctl->tol;
        tol_upd = ctl->tol_update;
        rho0 = ctl->rho0;
        if (k >= 4 && k < 256) {
            h1 = ctl->hist[k - 1];
            h2 = ctl->hist[k - 2];
            h3 = ctl->hist[k - 3];
            dh3 = ctl->dhist[k - 3];
        }
    }
    double A, B, D = 0.0, W = 0.0;
    reduce_pairs(partials, np, A, B);
    const bool upd = ndp > 0 && ctl->iter > 0 && ctl->tol_update > 0.0;
    __syncthreads();
    if (upd) reduce_pairs(dpart, ndp, D, W);
    if (threadIdx.x == 0) {
        const double rho = bn > 0.0 ? sqrt(A) / bn : sqrt(A);
        ctl->sum_r2 = A;
        ctl->sum_u2 = B;
        ctl->rho = rho;
        ctl->jbar = 3.0 * B * inv_dof;
        if (k < 256) ctl->hist[k] = rho;
        if (k == 0) {
            ctl->rho0 = rho;
            rho0 = rho;
        }
        // stagnation: no decrease over the last three corrections (the residual
        // sits at the rounding floor of the iterate's precision)
        const double dn = upd ? (W > 0.0 ? sqrt(D / W) : sqrt(D)) : 1.0;
        ctl->dnorm = dn;
        if (k < 256) ctl->dhist[k] = dn;
        // with the update-size test on, a still-shrinking correction is progress too
        const bool d_stalled = !upd || (k >= 4 && dn >= 0.99 * dh3);
        const bool stalled = k >= 4 && k < 256 && rho >= 0.99 * h3 && d_stalled;
        // divergence: monotone growth over the last three corrections and 10x overall
        // (a single jump can be rounding noise at the residual floor)
        const bool growing = k >= 4 && k < 256 && rho > 10.0 * h3 && rho > h1 && h1 > h2 && h2 > h3;
        int status = ST_RUNNING;
        if (!(rho == rho) || rho > 1e300 || (k > 0 && rho > 1e6 * rho0) || growing) status = -5;  // PINT_EDIVERGED
        else if (rho <= tol || (upd && dn <= tol_upd)) status = 0;                                // PINT_OK
        else if (k >= max_iter || stalled) status = -4;                                           // PINT_ENOCONV
        if (status == ST_RUNNING) ctl->iter = k + 1;
        else ctl->status = status;
        if (use_cond) cudaGraphSetConditional(cond, status == ST_RUNNING ? 1u : 0u);
    }
}

// Plain reduction for pint_residual: ctl->rho = sqrt(sum r^2)/bnorm, status untouched.
__global__ void __launch_bounds__(256) k_residual_norm(const double* __restrict__ partials, int np, Ctl* ctl) {
    double A, B;
    reduce_pairs(partials, np, A, B);
    if (threadIdx.x == 0) {
        const double bn = ctl->bnorm;
        ctl->sum_r2 = A;
        ctl->rho = bn > 0.0 ? sqrt(A) / bn : sqrt(A);
    }
}

// First iteration from U = 0: S[k][p] = u0[p]/dt for every k (the transform of
// b = (u0/dt, 0, ..., 0) with gamma_0 = 1); rho_0 = ||b||/||b|| = 1.
template <class T>
__global__ void k_zero_start(c_t<T>* __restrict__ S, const double* __restrict__ u0, double inv_dt, int nspace,
                             int nk, Ctl* __restrict__ ctl) {
    if (ctl->status != ST_RUNNING) return;
    const size_t total = (size_t)nspace * nk;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        S[i] = mkc((T)(u0[i % nspace] * inv_dt), T(0));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rho = ctl->bnorm > 0.0 ? 1.0 : 0.0;
        ctl->hist[0] = rho;
        ctl->rho0 = rho;
        ctl->rho = rho;
        ctl->jbar = 0.0;
        if (rho <= ctl->tol) ctl->status = 0;
        else ctl->iter = 1;
    }
}

__global__ void k_set_running(Ctl* ctl, double jbar) {
    ctl->status = ST_RUNNING;
    ctl->jbar = jbar;
}

// U[n][p] = u0[p] for all n.
__global__ void k_broadcast(double* __restrict__ U, const double* __restrict__ u0, int nspace, int nt) {
    size_t total = (size_t)nspace * nt;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        U[i] = u0[i % nspace];
}

// s[n][p] = (TS)(gamma_n r[n][p])  (the alpha-scaling of Step 1 for pint_precond_apply)
template <class TS>
__global__ void k_scale_cast(const double* __restrict__ r, const double* __restrict__ gam, TS* __restrict__ s,
                             int nspace, int nt) {
    size_t total = (size_t)nspace * nt;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        s[i] = (TS)(gam[i / nspace] * r[i]);
}

// Cahn-Hilliard invariants of each time level of a window (Sec. 1, Eq. 1.5),
// one CTA per level, deterministic (fixed per-thread order and tree):
//   out[2n]     = h^d sum_i u_i                                   (mass)
//   out[2n + 1] = h^d sum_i (u_i^2 - 1)^2 / 4
//                 + (eps^2 / 2) h^(d-2) sum over interior faces (u_j - u_i)^2   (discrete energy)
// U is FP64, or float-float (hi, lo) for the PINT_MIXED_FF iterate.
__device__ __forceinline__ double inv_val(const double* U, size_t i) { return U[i]; }
__device__ __forceinline__ double inv_val(const float2* U, size_t i) {
    const float2 v = U[i];
    return (double)v.x + (double)v.y;
}
template <class T>
__global__ void __launch_bounds__(256) k_invariants(const T* __restrict__ U, int nx, int ny, int dim, double hd,
                                                    double gcoef, double* __restrict__ out) {
    __shared__ double rm[8], re[8], rg[8];
    const int n = blockIdx.x;
    const size_t ns = (size_t)nx * (dim == 2 ? ny : 1);
    const T* u = U + (size_t)n * ns;
    double m = 0.0, e = 0.0, gsum = 0.0;
    for (size_t i = threadIdx.x; i < ns; i += 256) {
        const double v = inv_val(u, i);
        const int x = (int)(i % nx);
        m += v;
        const double w = v * v - 1.0;
        e = fma(0.25 * w, w, e);
        if (x + 1 < nx) {
            const double d = inv_val(u, i + 1) - v;
            gsum = fma(d, d, gsum);
        }
        if (dim == 2 && i + nx < ns) {
            const double d = inv_val(u, i + nx) - v;
            gsum = fma(d, d, gsum);
        }
    }
    m = warp_sum(m);
    e = warp_sum(e);
    gsum = warp_sum(gsum);
    if (threadIdx.x % 32 == 0) {
        rm[threadIdx.x / 32] = m;
        re[threadIdx.x / 32] = e;
        rg[threadIdx.x / 32] = gsum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = 0.0, Eb = 0.0, G = 0.0;
        for (int w = 0; w < 8; ++w) { M += rm[w]; Eb += re[w]; G += rg[w]; }
        out[2 * n] = hd * M;
        out[2 * n + 1] = hd * Eb + gcoef * G;
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
int residual_grid(const Geo& g, int& gx, int& gy, int& gz, int& chunk) {
    const int TX = g.dim == 2 ? 32 : 256, TY = g.dim == 2 ? 8 : 1;
    gx = (g.nx + TX - 1) / TX;
    gy = g.dim == 2 ? (g.ny + TY - 1) / TY : 1;
    const long tiles = (long)gx * gy;
    // enough CTAs for ~4 waves of 152 SMs, at least 4 time levels per CTA
    long want = (608 + tiles - 1) / tiles;
    chunk = (int)((g.nt + want - 1) / want);
    if (chunk < 4) chunk = 4;
    if (chunk > g.nt) chunk = g.nt;
    gz = (g.nt + chunk - 1) / chunk;
    return gx * gy * gz;
}

template <class TS>
void launch_residual(const Geo& g, const double* U, const double* u0, const double* gam, double* r_out, TS* s_out,
                     double* partials, const Ctl* ctl, cudaStream_t st) {
    int gx, gy, gz, chunk;
    residual_grid(g, gx, gy, gz, chunk);
    dim3 grid(gx, gy, gz);
    if (g.dim == 2)
        k_residual<2, TS><<<grid, 256, 0, st>>>(g, U, u0, gam, r_out, s_out, partials, ctl, chunk);
    else
        k_residual<1, TS><<<grid, 256, 0, st>>>(g, U, u0, gam, r_out, s_out, partials, ctl, chunk);
}
template void launch_residual<float>(const Geo&, const double*, const double*, const double*, double*, float*,
                                     double*, const Ctl*, cudaStream_t);
template void launch_residual<double>(const Geo&, const double*, const double*, const double*, double*, double*,
                                      double*, const Ctl*, cudaStream_t);

int norm2_blocks(int n) {
    int b = (n + 255) / 256;
    return b > 1024 ? 1024 : (b < 1 ? 1 : b);
}
void launch_begin_window(const Geo& g, const double* u0, int max_iter, double tol, double* partials, Ctl* ctl,
                         cudaStream_t st, double tol_update, double* b1) {
    if (g.th < 1.0 || g.expl) {
        // b_1 = u0/dt - (1-theta) A(u0) (Eyre: u0/dt - Lap u0): the first level of the residual at U = 0
        Geo g1 = g;
        g1.nt = 1;
        int gx, gy, gz, chunk;
        const int np = residual_grid(g1, gx, gy, gz, chunk);
        launch_residual<double>(g1, nullptr, u0, nullptr, b1, nullptr, partials, nullptr, st);
        k_begin_window<<<1, 256, 0, st>>>(partials, np, 1.0, max_iter, tol, tol_update, ctl);
        return;
    }
    int nb = norm2_blocks(g.nspace);
    k_norm2<<<nb, 256, 0, st>>>(u0, g.nspace, partials);
    k_begin_window<<<1, 256, 0, st>>>(partials, nb, g.inv_dt, max_iter, tol, tol_update, ctl);
}
void launch_after_residual(const double* partials, int np, double inv_dof, Ctl* ctl, cudaStream_t st,
                           unsigned long long cond, int use_cond, const double* dpart, int ndp) {
    launch_pdl(k_after_residual, dim3(1), dim3(256), 0, st, partials, np, inv_dof, ctl, (cudaGraphConditionalHandle)cond,
               use_cond, dpart, ndp);
}
void launch_residual_norm(const double* partials, int np, Ctl* ctl, cudaStream_t st) {
    k_residual_norm<<<1, 256, 0, st>>>(partials, np, ctl);
}
void launch_set_running(Ctl* ctl, double jbar, cudaStream_t st) { k_set_running<<<1, 1, 0, st>>>(ctl, jbar); }
void launch_broadcast(double* U, const double* u0, int nspace, int nt, cudaStream_t st) {
    size_t total = (size_t)nspace * nt;
    int nb = (int)((total + 255) / 256);
    if (nb > 4 * 152 * 8) nb = 4 * 152 * 8;
    k_broadcast<<<nb, 256, 0, st>>>(U, u0, nspace, nt);
}
template <class T>
void launch_zero_start(c_t<T>* S, const double* u0, double inv_dt, int nspace, int nk, Ctl* ctl, cudaStream_t st) {
    size_t total = (size_t)nspace * nk;
    int nb = (int)((total + 255) / 256);
    if (nb > 4 * 152 * 8) nb = 4 * 152 * 8;
    k_zero_start<T><<<nb, 256, 0, st>>>(S, u0, inv_dt, nspace, nk, ctl);
}
template void launch_zero_start<float>(float2*, const double*, double, int, int, Ctl*, cudaStream_t);
template void launch_zero_start<double>(double2*, const double*, double, int, int, Ctl*, cudaStream_t);

template <class TS>
void launch_scale_cast(const double* r, const double* gam, TS* s, int nspace, int nt, cudaStream_t st) {
    size_t total = (size_t)nspace * nt;
    int nb = (int)((total + 255) / 256);
    if (nb > 4 * 152 * 8) nb = 4 * 152 * 8;
    k_scale_cast<TS><<<nb, 256, 0, st>>>(r, gam, s, nspace, nt);
}
template void launch_scale_cast<float>(const double*, const double*, float*, int, int, cudaStream_t);
template void launch_scale_cast<double>(const double*, const double*, double*, int, int, cudaStream_t);

template <class T>
void launch_invariants(const T* U, int nlev, const Geo& g, double eps, double h, double* out, cudaStream_t st) {
    if (nlev <= 0) return;
    const double hd = g.dim == 2 ? h * h : h;
    const double gcoef = 0.5 * eps * eps * (g.dim == 2 ? 1.0 : 1.0 / h);   // (eps^2/2) h^(d-2)
    k_invariants<T><<<nlev, 256, 0, st>>>(U, g.nx, g.ny, g.dim, hd, gcoef, out);
}
template void launch_invariants<double>(const double*, int, const Geo&, double, double, double*, cudaStream_t);
template void launch_invariants<float2>(const float2*, int, const Geo&, double, double, double*, cudaStream_t);

}  // namespace pint
