// k_residual_ff.cu - the all-at-once residual in float-float arithmetic (about
// 48 significant bits on the FP32 pipes) for the PINT_MIXED_FF precision, plus
// the conversions between FP64 and float-float iterates.
//
// Same operator and boundary treatment as k_residual.cu (Eq. 2.6 / 4.8 with
// alpha = 0, theta = 1):
//   r_n = (u_{n-1} - u_n)/dt - [c2 Lap^2 u_n + c1 Lap u_n + cN Lap(u_n^3)].
// Every stencil sum is an accurate double-word addition, so the cancellation
// in the differences of smooth data costs no accuracy beyond ~2^-47 of the
// result.  Output: s = gamma_n r_n rounded to FP32 (the alpha-scaled input of
// Step 1), and per-CTA partial sums of r^2 and u^2.
#include "ff.cuh"
#include "pint_common.cuh"
#include "pint_kernels.h"

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

template <int DIM> struct ResTileFF;
template <> struct ResTileFF<1> { static constexpr int TX = 256, TY = 1; };
template <> struct ResTileFF<2> { static constexpr int TX = 32, TY = 8; };

template <int DIM>
__global__ void __launch_bounds__(256) k_residual_ff(GeoFF g, const ff* __restrict__ U, const ff* __restrict__ u0,
                                                     const float* __restrict__ gamf, float* __restrict__ s_out,
                                                     double* __restrict__ partials, const Ctl* __restrict__ ctl,
                                                     int chunk) {
    if (ctl && ctl->status != ST_RUNNING) return;
    constexpr int TX = ResTileFF<DIM>::TX, TY = ResTileFF<DIM>::TY;
    constexpr int HY = DIM == 2 ? 2 : 0;
    constexpr int SX = TX + 4, SY = TY + 2 * HY;
    constexpr int LX = TX + 2, LY = TY + (DIM == 2 ? 2 : 0);
    __shared__ ff su[SY * SX];
    __shared__ ff sL[LY * LX];
    __shared__ double red[2][8];

    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool inside = gx < g.nx && (DIM == 1 || gy < g.ny);
    const int pidx = (DIM == 2 ? gy * g.nx : 0) + gx;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(g.nt, n0 + chunk);
    const bool ch = g.cN != 0.f;
    const bool lin1 = g.c1.x != 0.f;

    ff uprev = ffmk(0.f, 0.f);
    if (inside) uprev = n0 == 0 ? u0[pidx] : U[(size_t)(n0 - 1) * g.nspace + pidx];
    float acc_r2 = 0.f, acc_u2 = 0.f;

    for (int n = n0; n < n1; ++n) {
        const ff* un = U + (size_t)n * g.nspace;
        for (int e = threadIdx.x; e < SX * SY; e += TX * TY) {
            int ix = e % SX, iy = e / SX;
            su[e] = ext_read_ff(un, x0 - 2 + ix, y0 - HY + iy, g.nx, g.ny, DIM, g.bc);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < LX * LY; e += TX * TY) {
            int ix = e % LX, iy = e / LX;
            const int c = (DIM == 2 ? (iy + 1) * SX : 0) + ix + 1;
            ff v = ff_mul(ff_d2(su[c - 1], su[c + 1], su[c]), g.ihx2);
            if (DIM == 2) v = ff_add(v, ff_mul(ff_d2(su[c - SX], su[c + SX], su[c]), g.ihy2));
            sL[e] = v;
        }
        __syncthreads();
        if (inside) {
            const int cl = (DIM == 2 ? (ty + 1) * LX : 0) + tx + 1;
            const int cu = (ty + HY) * SX + tx + 2;
            const ff L = sL[cl];
            ff L2 = ff_mul(ff_d2(sL[cl - 1], sL[cl + 1], L), g.ihx2);
            if (DIM == 2) L2 = ff_add(L2, ff_mul(ff_d2(sL[cl - LX], sL[cl + LX], L), g.ihy2));
            const ff u = su[cu];
            ff A = ff_mul(L2, g.c2);
            if (lin1) A = ff_add(A, ff_mul(L, g.c1));
            if (ch) {  // cN = -1: A -= Lap(u^3)
                const ff w0 = ff_cube(u);
                ff lw = ff_mul(ff_d2(ff_cube(su[cu - 1]), ff_cube(su[cu + 1]), w0), g.ihx2);
                if (DIM == 2) lw = ff_add(lw, ff_mul(ff_d2(ff_cube(su[cu - SX]), ff_cube(su[cu + SX]), w0), g.ihy2));
                A = ff_sub(A, lw);
            }
            const ff r = ff_sub(ff_mul(ff_sub(uprev, u), g.inv_dt), A);
            const float gm = gamf[n];
            s_out[(size_t)n * g.nspace + pidx] = fmaf(gm, r.x, gm * r.y);
            acc_r2 = fmaf(r.x, r.x, acc_r2);
            acc_u2 = fmaf(u.x, u.x, acc_u2);
            uprev = u;
        }
        __syncthreads();
    }
    double a = warp_sum((double)acc_r2), b = warp_sum((double)acc_u2);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) { red[0][warp] = a; red[1][warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, B = 0.0;
        for (int w = 0; w < (TX * TY) / 32; ++w) { A += red[0][w]; B += red[1][w]; }
        size_t cta = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[2 * cta] = A;
        partials[2 * cta + 1] = B;
    }
}

__global__ void k_f64_to_ff(const double* __restrict__ in, ff* __restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = ff_from_double(in[i]);
}
__global__ void k_ff_to_f64(const ff* __restrict__ in, double* __restrict__ out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const ff v = in[i];
        out[i] = (double)v.x + (double)v.y;
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

void launch_residual_ff(const GeoFF& g, const Geo& g64, const ff* U, const ff* u0, const float* gamf, float* s,
                        double* partials, const Ctl* ctl, cudaStream_t st) {
    int gx, gy, gz, chunk;
    residual_grid(g64, gx, gy, gz, chunk);
    dim3 grid(gx, gy, gz);
    if (g.dim == 2) k_residual_ff<2><<<grid, 256, 0, st>>>(g, U, u0, gamf, s, partials, ctl, chunk);
    else k_residual_ff<1><<<grid, 256, 0, st>>>(g, U, u0, gamf, s, partials, ctl, chunk);
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
