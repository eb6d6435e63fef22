// pint_kernels.h - host-side launchers of the libpint kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fx.cuh"
#include "pint_common.cuh"

namespace pint {

// Device tables of one problem in the transform precision T.
template <class T> struct Tabs {
    const c_t<T>* twt;   // nt:  exp(-2 pi i j / nt)
    const c_t<T>* twx;   // nx:  exp(-2 pi i j / nx)          (FFT cosine path)
    const c_t<T>* twy;   // ny
    const c_t<T>* wx;    // nx:  exp(-i pi p / (2 nx))        (DCT-II post-twiddle)
    const c_t<T>* wy;    // ny
    const T* fx;         // nx*nx dense forward basis [p][j]  (dense path)
    const T* ix;         // nx*nx dense inverse basis [j][p]
    const T* fy;         // ny*ny
    const T* iy;         // ny*ny
    const c_t<T>* dsx;   // 2(nx+1): exp(-2 pi i j / (2(nx+1)))   (sine path)
    const c_t<T>* dsy;   // 2(ny+1)
    const T* lamx;       // nx:  eigenvalues of the 1-D Laplacian along x
    const T* lamy;       // ny
    const c_t<T>* lam1;  // nt/2+1: lambda_1k of Lemma 2.1
    const c_t<T>* lam2;  // nt/2+1: lambda_2k
    T dte;               // Eyre splitting (PinT-II): dt, so that lambda_3k = 1 - dt lambda_1k; else 0
};

// Coefficients of the shifted spatial solve: mu(Lam) = c2 Lam^2 + c1 Lam,
// c1 - jbar (jbar read from ctl) when ch != 0: 1 - jbar for PinT-I, -jbar
// for PinT-II (whose explicit Laplacian enters as lambda_3k Lam).
struct SolveCoef {
    double c2, c1;
    int ch;
};

// Float-float form of Geo for the PINT_MIXED_FF residual (constants as hi + lo
// pairs).  c2, c1, cN carry the factor dt (the residual is evaluated as
// dt r); on square cells (and in 1-D) the stencil sums are unscaled and they
// also carry the factors 1/h^4, 1/h^2, 1/h^2.
struct GeoFF {
    int nx, ny, dim, bc, nt, nspace;
    float2 ihx2, ihy2, inv_dt, c2, c1, cN;
    int accurate;   // 1: chained accurate double-word stencil sums (very stiff problems)
    int half;       // theta = 1/2: the residual also carries A'(u_{n-1})
    int expl;       // Eyre splitting: the c1 Laplacian term acts on u_{n-1}
};

// Geometry of the block fixed-point residual (k_residual_fx.cu): the products
// dt c1 / h^2 and dt c2 / h^4 as integer mantissas in one binary frame.
struct GeoFX {
    int nx, ny, dim, bc, nt, nspace;
    int half;       // theta = 1/2: A(u_{n-1}) enters too
    int lin1;       // c1 != 0 (the Laplacian term is present)
    int neg1;       // c1 < 0 (signed beta^2)
    int cube;       // cN != 0 (Cahn-Hilliard: the Lap(u^3) term)
    int negN;       // cN < 0
    int Q;          // exponent of the largest coefficient's frame
    int dQ1, dQ2, dQN;       // |c_i| = M_i 2^(Q - dQ_i)
    int bM1, bM2, bMN;       // significant bits of M_i (53, or 0 for an absent term)
    int64_t M1, M2, MN;      // the coefficients' 53-bit mantissas
    double inv_dt;
};
// Linear equations (theta 1 or 1/2) and Cahn-Hilliard PinT-I (theta 1), square cells or 1-D.
int residual_fx_supported(const Geo& g);
GeoFX make_geo_fx(const Geo& g);
int residual_fx_grid(const Geo& g, int& gx, int& gy, int& gz, int& chunk);
// rout_mode 0: s = gamma_n r rounded to FP32 (gdt[n] = gamma_n / dt, igamf[n] = 1/gamma_n);
// rout_mode 1: r in FP64 into r_out (may be nullptr: norm only; s, gdt, igamf unused).
// Per-CTA (sum r^2, 0) pairs in partials.
cudaError_t launch_residual_fx(const GeoFX& f, const Geo& g, const double* U, const double* u0, const double* gdt,
                               const float* igamf, float* s, double* r_out, double* partials, const Ctl* ctl,
                               cudaStream_t st, int rout_mode);

// Factorization of a long time axis (N_t > 1024) for the multi-pass FFT of
// k_timefft.cu: N_t = f_0 ... f_{S-1}, istr_s = prod_{j>s} f_j,
// P_s = prod_{j<s} f_j, all powers of two (lf, listr, lP their logarithms).
struct LongPlan {
    int S;
    int f[3], istr[3], P[3];
    int lf[3], listr[3], lP[3];
};
LongPlan long_plan(int nt);
#ifdef __CUDACC__
// Workspace row of Z_k after the last forward pass: sum_s k_s istr_s, k = sum_s k_s P_s.
__device__ __forceinline__ int long_pos(int k, const LongPlan& pl) {
    int r = 0;
    for (int i = 0; i < pl.S; ++i) r += ((k >> pl.lP[i]) & (pl.f[i] - 1)) << pl.listr[i];
    return r;
}
#endif
// 1-D long axes: the spatial solve of Step 2 done by the pack of the inverse
// time transform (one pass over the half spectrum instead of two).
template <class T> struct LongSolve {
    const Tabs<T>* tb;
    SolveCoef co;
    int nx;
};
// Rows of N = nx points on the cosine (FFT) path: S[k] solved and written as the pack
// workspace rows z[long_pos(k)], z[long_pos(N_t - k)] (k = 0..N_t/2).
template <class T>
cudaError_t launch_long_pack_solve(int nt, const c_t<T>* S, c_t<T>* z, const LongSolve<T>& ls, const Ctl* ctl,
                                   cudaStream_t st);

int residual_grid(const Geo& g, int& gx, int& gy, int& gz, int& chunk);
int residual_ff_grid(const Geo& g, int& gx, int& gy, int& gz, int& chunk);
void launch_residual_ff(const GeoFF& g, const Geo& g64, const float2* U, const float2* u0, const float* gamf,
                        float* s, double* partials, const Ctl* ctl, cudaStream_t st);
void launch_f64_to_ff(const double* in, float2* out, size_t n, cudaStream_t st);
void launch_ff_to_f64(const float2* in, double* out, size_t n, cudaStream_t st);
void launch_broadcast_ff(float2* U, const float2* u0, int nspace, int nt, cudaStream_t st);
cudaError_t launch_time_inv_ff(int nt, int nspace, const float2* S, const float2* twt, const float* ginvf,
                               float2* Uff, const Ctl* ctl, double* dpart, cudaStream_t st, void* work = nullptr,
                               const LongSolve<float>* ls = nullptr);
template <class TS>
void launch_residual(const Geo& g, const double* U, const double* u0, const double* gam, double* r_out, TS* s_out,
                     double* partials, const Ctl* ctl, cudaStream_t st);
int norm2_blocks(int n);
// Window start: ||b|| into ctl->bnorm and the iteration state reset.  theta < 1
// computes b_1 = u0/dt - (1-theta) A u0 (stored in b1 when b1 != nullptr).
void launch_begin_window(const Geo& g, const double* u0, int max_iter, double tol, double* partials, Ctl* ctl,
                         cudaStream_t st, double tol_update = 0.0, double* b1 = nullptr);
// cond / use_cond: CUDA-graph while-loop condition handle (see pint_api.cu).
// dpart/ndp: the last correction's (sum delta^2, sum U^2) partials (ndp = 0: none).
void launch_after_residual(const double* partials, int np, double inv_dof, Ctl* ctl, cudaStream_t st,
                           unsigned long long cond = 0, int use_cond = 0, const double* dpart = nullptr,
                           int ndp = 0);
void launch_residual_norm(const double* partials, int np, Ctl* ctl, cudaStream_t st);
void launch_set_running(Ctl* ctl, double jbar, cudaStream_t st);
void launch_broadcast(double* U, const double* u0, int nspace, int nt, cudaStream_t st);
template <class TS>
void launch_scale_cast(const double* r, const double* gam, TS* s, int nspace, int nt, cudaStream_t st);

// Step 1: S[k] = sum_n s[n] exp(-2 pi i nk/nt), k = 0..nt/2 (s already alpha-scaled).
template <class T>
cudaError_t launch_time_fwd(int nt, int nspace, const T* s, c_t<T>* S, const c_t<T>* twt, const Ctl* ctl,
                            cudaStream_t st);
// Step 3: delta_n = ginv[n] * Re( sum_k S[k] exp(+2 pi i nk/nt) ) over the full
// Hermitian spectrum; U += delta (accumulate) or out = delta.
// dpart (may be NULL): per-CTA (sum delta^2, sum U^2) pairs, time_inv_blocks() of them.
// ls (N_t > 1024, 1-D, may be NULL): solve Step 2 on the way (S then holds the unsolved spectrum).
template <class T>
cudaError_t launch_time_inv(int nt, int nspace, const c_t<T>* S, const c_t<T>* twt, const double* ginv, double* out,
                            int accumulate, const Ctl* ctl, double* dpart, cudaStream_t st, void* work = nullptr,
                            const LongSolve<T>* ls = nullptr);
int time_inv_blocks(int nt, int nspace, int f32);
// Kernel launches of one forward / inverse time transform (several passes beyond 1024 steps).
int time_fwd_launches(int nt);
int time_inv_launches(int nt);

// Vector kernels of the outer flexible GMRES (k_krylov.cu).  At most
// kMaxKrylov basis vectors per restart.
constexpr int kMaxKrylov = 30;
int krylov_dot_blocks(size_t n);
// partials[b * nv + i]: CTA b's part of w . v_i for v_i = V + i * ld, i < nv (krylov_dot_blocks(n) CTAs)
void launch_multi_dot(const double* w, const double* V, size_t ld, int nv, size_t n, double* partials,
                      cudaStream_t st);
// w += sum_i c[i] v_i (c on the device)
void launch_multi_axpy(double* w, const double* V, size_t ld, int nv, const double* c, size_t n, cudaStream_t st);
void launch_scale_copy(double* y, const double* x, double a, size_t n, cudaStream_t st);

// Space-varying averaged Jacobian and the inner solve of Step 2 (k_jacobian.cu).
// Every vector kernel below takes an optional device flag `skip`: when it is
// nonzero at launch the kernel does nothing (the inner cycle has stopped), so
// that one fixed launch sequence serves every cycle and can be captured.
template <class T>
void launch_jtilde(const double* U, const float2* uff, int nt, int nspace, T* jt, cudaStream_t st);
// W[k] = lambda_1k Y[k] + lambda_2k (c2 Lap^2 Y[k] + Lap((c1 - J~) Y[k])) + lambda_3k Lap Y[k], k < nk
// (W = B - that, when B is given)
template <class T>
void launch_apply_M(const Geo& g, int nk, const c_t<T>* Y, c_t<T>* W, const T* jt, const Tabs<T>& tb, double c2,
                    double c1, const int* skip, const c_t<T>* B, cudaStream_t st);
// Device state of the inner flexible GMRES: a head shared by the cycle and one
// block per frequency slice (the operator is block-diagonal over the slices,
// so each gets its own Krylov coefficients; classical Gram-Schmidt with a
// conditional second pass, complex Givens rotations, FP64 scalars).  The small
// kernels below update it from the dot products' per-CTA partials, which they
// add in a fixed order, so the cycle is deterministic and needs no host round trip.
struct GmHead {
    Ctl ictl;                 // control word of the cycle's spatial solves: jbar, status ST_RUNNING while it runs
    int skip;                 // nonzero once every slice has left the cycle (or the outer iteration has stopped)
    int ndone;                // slices that have left
    int jmax;                 // steps run
    int skip_re[kMaxKrylov];  // step j's second Gram-Schmidt pass is skipped unless a slice asked for it
};
struct GmK {
    int done, reorth, j, pad;
    double bn, hn2, scale;    // ||S1_k||; the norm^2 estimate of the new vector; its normalization factor
    double cs[kMaxKrylov];
    double2 sn[kMaxKrylov];
    double2 gv[kMaxKrylov + 1];
    double2 H[kMaxKrylov * kMaxKrylov];   // upper triangle, row i, column j at i * kMaxKrylov + j
    double2 hcol[kMaxKrylov + 1];
    double2 coef[kMaxKrylov + 1];        // projection coefficients of the step's last pass
    double2 coefA[kMaxKrylov + 1];       // those of its first pass when a second one follows, else 0
    double2 y[kMaxKrylov];               // the solution of the cycle's least-squares problem
    double2 tmp[kMaxKrylov + 2];
};
// CTAs per slice (x) of the per-slice vector kernels.
int cdot_blocks(size_t ns, int nk);
// partials[((k nbx + bx) nv + i) 2 + {re, im}] of <v_i, w> on slice k, nbx = cdot_blocks(ns, nk)
template <class T>
void launch_cmulti_dot(const c_t<T>* w, const c_t<T>* V, size_t ld, int nv, size_t ns, int nk, double* partials,
                       const int* skip, cudaStream_t st);
// Which coefficients of GmK the axpy reads: coef, coefA, y.
enum { GM_COEF = 0, GM_COEFA = 1, GM_Y = 2 };
// out = (w + sum_{i < min(nv, nlim, *nlimd)} c_{k,i} v_i) * (post ? scale_k : 1) on each slice k
// (out = w when null; nlimd optional; nv = 0: the scaling alone)
template <class T>
void launch_cmulti_axpy(c_t<T>* w, const c_t<T>* V, size_t ld, int nv, int nlim, size_t ns, int nk, const GmK* gk,
                        int sel, const int* skip, cudaStream_t st, c_t<T>* out = nullptr, int post = 0,
                        const int* nlimd = nullptr);
// z = a x + b y (y may be null); with sdev, a is *sdev instead
template <class T>
void launch_caxpby(c_t<T>* z, double a, const c_t<T>* x, double b, const c_t<T>* y, size_t n, const int* skip,
                   const double* sdev, cudaStream_t st);
void launch_gm_reset(GmHead* h, cudaStream_t st);
// Start: ||S1_k|| and ||r0_k|| from two single-vector partial sets; a slice with
// ||r0_k|| <= tol ||S1_k|| (or every slice, when the outer iteration has stopped) leaves at once.
void launch_gm_init(const double* part_bb, const double* part_rr, int nbx, const Ctl* octl, GmHead* h, GmK* gk,
                    int nk, double tol, cudaStream_t st);
// Step j, first pass: h_i = <v_i, w>, i <= j, and <w, w> from partials of j + 2 vectors.
void launch_gm_orth1(const double* part, int nbx, int j, GmHead* h, GmK* gk, int nk, cudaStream_t st);
// Step j, second pass (if taken), the norm, the rotations and the stop test.
void launch_gm_orth2(const double* part, int nbx, int j, GmHead* h, GmK* gk, int nk, double tol, cudaStream_t st);
// y_k = H_k^{-1} g_k over slice k's completed steps.
void launch_gm_solve(GmK* gk, int nk, cudaStream_t st);
// CTAs of launch_time_inv_ff (with the same control block argument).
int time_inv_ff_blocks(int nt, int nspace, const Ctl* ctl);
// Step 2: per frequency k, S[k] <- (lambda_1k I + lambda_2k A)^{-1} S[k], in
// stages: 1-D: stage 0 = fused transform/divide/inverse along x.  2-D: stage 0
// = forward along x, 1 = fused along y (with the division), 2 = inverse along x.
template <class T>
cudaError_t launch_spatial_stage(int stage, const Geo& g, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, int fft_x,
                                 int fft_y, const Ctl* ctl, cudaStream_t st);

// First iteration from the zero iterate: r = b = (u0/dt, 0, ..., 0), so the
// alpha-scaled time transform is u0/dt at every frequency.  Writes S and
// records rho_0 = 1 in ctl (or stops if tol >= 1).
template <class T>
void launch_zero_start(c_t<T>* S, const double* u0, double inv_dt, int nspace, int nk, Ctl* ctl, cudaStream_t st);

// Fused 2-D solve of every frequency slice in one kernel (thread-block cluster
// per slice); for square grids of 64, 128 (FP32/FP64) or 256 (FP32) cells per side.
int slice2d_supported(const Geo& g, int fft_x, int fft_y, int f32);
// Sine path of a simply supported axis of n points: n + 1 a power of two, 3 <= n <= 4095.
int dst_axis_supported(int n);
// Project autotuner table (tune_cache.cu): per problem shape, the transform
// choices measured fastest on this device.  Thread-safe; PINT_TUNE_FILE names a
// text file loaded at the first lookup and appended to by every new entry.
struct TuneKey {
    int equation, dim, nx, ny, nt, precision, bc, half;
};
struct TuneVal {
    int gemm_fwd, gemm_inv, fused;   // 1: tensor-core DFT for Step 1 / Step 3; one-kernel 2-D Step 2
    float ms;                        // measured time of the chosen combination
};
bool tune_lookup(const TuneKey& k, TuneVal* v);
void tune_store(const TuneKey& k, const TuneVal& v);
int tune_load(const char* path);   // entries read; -1: no such file; -2: malformed line (entries before it kept)
int tune_save(const char* path);   // entries written, or -1
void tune_clear();
// Shared-memory attributes and resident-CTA counts of the sine-path kernels of
// an axis of n points (axis 0: rows, 1: columns; f32: complex64 transforms).
// Called outside any stream capture before the first launch.
cudaError_t configure_dst(int n, int axis, int f32);
template <class T>
cudaError_t launch_slice2d(const Geo& g, c_t<T>* S, const Tabs<T>& tb, SolveCoef co, const Ctl* ctl,
                           cudaStream_t st);

// Per-level Cahn-Hilliard mass and discrete energy (Eq. 1.5) of nlev levels of U
// (FP64 or float-float), one (mass, energy) pair per level into out.
template <class T>
void launch_invariants(const T* U, int nlev, const Geo& g, double eps, double h, double* out, cudaStream_t st);

// Steps 1 and 3 as DFT matrix products on the tensor cores (k_timegemm.cu), for
// N_t = 64 or 128 and a point count divisible by 4.  Tables: FP16 hi and lo parts of
// the forward and inverse matrices (time_gemm_tables).  inv = 0: src = s (FP32
// [n][p]), dst = S (complex64 half spectrum); inv = 1: src = S, dst = U (FP64),
// U += gamma^{-1} x / N_t, with (sum delta^2, sum U^2) per CTA in dpart (may be NULL).
int time_gemm_supported(int nt, int nspace);
int time_gemm_blocks(int nspace);
void time_gemm_tables(int nt, std::vector<uint16_t>& out);
cudaError_t launch_time_gemm(int inv, int nt, int nspace, const void* src, void* dst, const void* wtab,
                             const double* ginv, Ctl* ctl, double* dpart, cudaStream_t st);

// Opt-in shared memory sizes for the kernels that need more than 48 KB.
cudaError_t configure_kernels();

}  // namespace pint
