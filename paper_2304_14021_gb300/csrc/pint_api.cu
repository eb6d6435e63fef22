// pint_api.cu - the C ABI of libpint (declared in include/pint.h): handle
// lifetime, host-built FP64 tables, and the outer iteration
//     U <- U + P_alpha^{-1} (b - K(U))
// (residual-correction form of the PinT iteration, Eq. 2.6-2.8; PinT-I of
// Eq. 4.11-4.14 for Cahn-Hilliard) driven from the host in chunks of
// iterations with a device-side status word, so the host reads back one small
// control block per chunk instead of synchronizing every iteration.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <complex>
#include <algorithm>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/pint.h"
#include "ff.cuh"
#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

template <class T> cudaError_t configure_time_all();
template <class T> cudaError_t configure_spatial_all();
cudaError_t configure_residual_ff();
cudaError_t configure_time_gemm();

cudaError_t configure_kernels() {
    static int done = -1;  // per process: the attributes are per device function
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorUnknown;
    if (done == dev) return cudaSuccess;
    cudaError_t e;
    if ((e = configure_time_all<float>()) != cudaSuccess) return e;
    if ((e = configure_time_all<double>()) != cudaSuccess) return e;
    if ((e = configure_spatial_all<float>()) != cudaSuccess) return e;
    if ((e = configure_spatial_all<double>()) != cudaSuccess) return e;
    if ((e = configure_residual_ff()) != cudaSuccess) return e;
    if ((e = configure_time_gemm()) != cudaSuccess) return e;
    done = dev;
    return cudaSuccess;
}

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Per-axis transform path: 1 = FFT-based cosine transform, 0 = dense basis.
// Transform path of one axis: 1 = cosine FFT (cell-centred Neumann, n a power
// of two up to nmax_fft), 2 = sine FFT (simply supported, n + 1 a power of two,
// 3 <= n <= 4095), 0 = dense basis tables (n <= 1024).
static int axis_fft(int n, int bc, int nmax_fft) {
    if (bc == PINT_BC_NEUMANN && is_pow2(n) && n >= 2 && n <= nmax_fft) return 1;
    if (bc == PINT_BC_SIMPLY_SUPPORTED && dst_axis_supported(n)) return 2;
    return 0;
}

static int validate(const pint_problem* p) {
    if (!p) return PINT_EINVAL;
    if (p->equation < 0 || p->equation > 3) return PINT_EINVAL;
    if (p->dim != 1 && p->dim != 2) return PINT_EINVAL;
    if (p->bc != PINT_BC_SIMPLY_SUPPORTED && p->bc != PINT_BC_NEUMANN && p->bc != PINT_BC_NEUMANN_VERTEX)
        return PINT_EINVAL;
    if (p->bc == PINT_BC_NEUMANN_VERTEX && (p->nx < 3 || (p->dim == 2 && p->ny < 3))) return PINT_EINVAL;
    if (p->nx < 2 || (p->dim == 2 && p->ny < 2)) return PINT_EINVAL;
    if (!is_pow2(p->nt) || p->nt < 2 || p->nt > (1 << 20)) return PINT_EINVAL;
    // time axes beyond 1024 steps take the four-step FFT, which pairs neighbouring spatial points
    if (p->nt > 1024 && ((long)p->nx * (p->dim == 2 ? p->ny : 1)) % 2 != 0) return PINT_EINVAL;
    if (p->n_windows < 1) return PINT_EINVAL;
    // theta-method: backward Euler (1) for every equation, Crank-Nicolson (1/2) for the linear ones
    const bool chq = p->equation == PINT_CAHN_HILLIARD || p->equation == PINT_CAHN_HILLIARD_EYRE;
    if (!(p->theta == 1.0 || (p->theta == 0.5 && !chq))) return PINT_EINVAL;
    if (!(p->alpha > 0.0 && p->alpha < 1.0)) return PINT_EINVAL;
    if (!(p->tol > 0.0) || !isfinite(p->tol)) return PINT_EINVAL;
    if (p->max_iter < 1 || p->max_iter >= PINT_HIST_MAX) return PINT_EINVAL;
    if (p->precision != PINT_FP64 && p->precision != PINT_MIXED && p->precision != PINT_MIXED_FF) return PINT_EINVAL;
    if (!(p->T > 0.0) || !isfinite(p->T)) return PINT_EINVAL;
    if (p->equation != PINT_BIHARMONIC && !(p->eps > 0.0)) return PINT_EINVAL;
    if (!isfinite(p->beta) || !isfinite(p->eps)) return PINT_EINVAL;
    if (p->init_guess < 0 || p->init_guess > 2) return PINT_EINVAL;
    if (!(p->tol_update >= 0.0) || !isfinite(p->tol_update)) return PINT_EINVAL;
    const int ny = p->dim == 2 ? p->ny : 1;
    if (!axis_fft(p->nx, p->bc, 4096) && p->nx > 1024) return PINT_EINVAL;
    if (p->dim == 2 && !axis_fft(ny, p->bc, 1024) && ny > 1024) return PINT_EINVAL;
    if ((long long)p->nx * ny > (1LL << 30)) return PINT_EINVAL;
    return PINT_OK;
}

static double grid_h(int n, int bc) {
    return bc == PINT_BC_SIMPLY_SUPPORTED ? 1.0 / (n + 1) : bc == PINT_BC_NEUMANN_VERTEX ? 1.0 / (n - 1) : 1.0 / n;
}

// Eigenvalue of the 1-D Delta_h for transform index p (Sec. 2.2 spectrum).
static double lap_eig(int p, int n, int bc) {
    const double h = grid_h(n, bc);
    const double s = bc == PINT_BC_SIMPLY_SUPPORTED ? sin(M_PI * (p + 1) / (2.0 * (n + 1)))
                     : bc == PINT_BC_NEUMANN_VERTEX  ? sin(M_PI * p / (2.0 * (n - 1)))
                                                     : sin(M_PI * p / (2.0 * n));
    return -4.0 / (h * h) * s * s;
}

static bool f32_transforms(const pint_problem* p) { return p->precision != PINT_FP64; }

// The first right-hand-side level b_1 involves u0 beyond u0/dt (theta < 1, or
// Eyre's explicit Laplacian): it is computed once per window and kept.
static bool needs_b1(const pint_problem* p) { return p->theta < 1.0 || p->equation == PINT_CAHN_HILLIARD_EYRE; }

// Pinned host mirrors of the device control blocks, carved from one page-locked
// slab per process (page-locking per handle would be slow and would serialize
// with work already running on the device).
static std::mutex g_slab_mu;
static Ctl* g_slab = nullptr;
static std::vector<Ctl*> g_slab_free;
static const int kSlabCtls = 1024;

static Ctl* ctl_slab_acquire() {
    std::lock_guard<std::mutex> lock(g_slab_mu);
    if (!g_slab) {
        if (cudaHostAlloc((void**)&g_slab, sizeof(Ctl) * kSlabCtls, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            g_slab = nullptr;
            return nullptr;
        }
        for (int i = kSlabCtls - 1; i >= 0; --i) g_slab_free.push_back(g_slab + i);
    }
    if (g_slab_free.empty()) return nullptr;
    Ctl* c = g_slab_free.back();
    g_slab_free.pop_back();
    return c;
}
static void ctl_slab_release(Ctl* c) {
    if (!c) return;
    std::lock_guard<std::mutex> lock(g_slab_mu);
    g_slab_free.push_back(c);
}

struct Sizes {
    size_t nspace, dof, nk, partials, tables_T, tables_bytes;
};

template <class T> struct Impl;

}  // namespace pint

struct pint_handle {
    pint_problem p;
    cudaStream_t st;
    int device = 0;                 // device current at pint_create
    int fft_x, fft_y;
    pint::Geo geo;
    pint::SolveCoef coef;
    pint::Ctl* ctl = nullptr;       // device
    pint::Ctl* hctl = nullptr;      // pinned host mirror
    double* partials = nullptr;
    int npart = 0;
    double* dpart = nullptr;        // per-CTA (sum delta^2, sum U^2) of the last correction
    double* gam = nullptr;          // alpha^{n/nt}
    double* ginv = nullptr;         // alpha^{-n/nt} / nt
    double* gdt = nullptr;          // PINT_MIXED: gamma_n / dt (the alpha-scaling of the fixed-point residual)
    float* igamf = nullptr;         // PINT_MIXED: 1 / gamma_n (its norm partials)
    pint::GeoFX gfx;                // block fixed-point residual geometry
    int use_fx = 0;                 // PINT_MIXED with the block fixed-point residual (linear, square cells)
    // time transforms as DFT matrix products on the tensor cores (k_timegemm.cu)
    int tgemm_mode = -1;            // -1: chosen by measurement on the first solve, 0: off, 1: on
    int gemm_fwd = 0, gemm_inv = 0; // in use for Step 1 / Step 3 (FP64 update)
    int tgemm_tuned = 0;
    void* wgemm = nullptr;          // FP16 DFT tables (hi, lo) of both directions for N_t = p.nt
    double* u0buf = nullptr;        // window initial condition
    double* b1 = nullptr;           // theta < 1: first right-hand-side level u0/dt - (1-theta) A u0
    double* hU = nullptr;           // pint_solve_host buffers (lazy)
    double* hu0 = nullptr;
    void* s = nullptr;              // alpha-scaled residual, transform precision
    void* S = nullptr;              // half spectrum, complex transform precision
    void* tab = nullptr;            // tables block
    // PINT_MIXED_FF: float-float iterate and its tables
    float2* Uff = nullptr;          // nt*nspace
    float2* Uff_cur = nullptr;      // first time level of the current segment within Uff
    float2* u0ff = nullptr;         // nspace
    float* gamf = nullptr;          // alpha^{n/nt} (FP32)
    float* ginvf = nullptr;         // alpha^{-n/nt}/nt (FP32)
    pint::GeoFF gff;
    long long bytes = 0;
    void* tabs_ptrs = nullptr;      // Tabs<T>* (host struct of device pointers)
    // profiling: launch counters always, event pairs around phases when enabled
    long long launches[PINT_NPHASE] = {0};
    double ms[PINT_NPHASE] = {0};
    int prof_on = 0;
    static const int NEV = 64;      // event pairs in the pool
    cudaEvent_t ev[2 * NEV] = {};
    int ev_phase[NEV] = {0};
    int nev = 0;
    // CUDA-graph execution of the iteration loop (one while-loop graph per window)
    int use_graphs = 1;
    int fuse2d = 1;                          // fused 2-D spatial kernel where supported
    int fuse2d_user = 0;                     // fuse2d set by the caller (not left to the autotuner)
    int tune_cached = 0;                     // the autotuner's choices came from its table
    int capturing = 0;                       // set while the loop body is being captured
    unsigned long long gcond = 0;            // cudaGraphConditionalHandle of the graph being captured
    cudaStream_t capst = nullptr;            // capture stream
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        const void* U = nullptr;
        const void* u0 = nullptr;
        unsigned long long cond = 0;
    } gslot[2];
    int gnext = 0;
    // time-axis levels (segment lengths nt, nt/2, ...) for the adaptive window policy
    struct Level {
        int nt = 0;
        void* tabs = nullptr;        // Tabs<T>* with twt, lam1, lam2 of this length
        double* gam = nullptr;
        double* ginv = nullptr;
        float* gamf = nullptr;
        float* ginvf = nullptr;
        double* gdt = nullptr;
        float* igamf = nullptr;
        void* block = nullptr;       // device block owning this level's tables (levels >= 1)
    } lev[11];
    int nlev = 0;
    int adaptive = 0;
    std::vector<double> lamx_h, lamy_h;   // host copies of the Laplacian eigenvalues
    // outer flexible GMRES (PINT_OPT_KRYLOV): restart length and FP64 work vectors
    int krylov = 0;
    double* kv = nullptr;      // (krylov + 1) basis vectors of nt * nspace
    double* kz = nullptr;      // krylov preconditioned vectors P^{-1} v_j
    double* kzero = nullptr;   // nspace zeros (the initial condition of K applied alone)
    double* kpart = nullptr;   // dot-product partial sums
    double* kcoef = nullptr;   // device copy of combination coefficients
    // space-varying Jacobian (PINT_OPT_VARYING_JACOBIAN): inner GMRES length and work vectors
    int vary = 0;
    void* jbuf = nullptr;      // solution, (vary + 1) basis and vary preconditioned spectra
    void* jt = nullptr;        // J~(x), one per spatial point
    double* jpart = nullptr;   // complex dot partial sums
    pint::GmHead* gmh = nullptr;     // device state of the inner GMRES cycle: head
    pint::GmK* gmk = nullptr;        //   and one block per frequency slice
    double vary_tol = 1e-4;    // relative residual of the inner solve
    // per-level invariants (PINT_OPT_LOG_INVARIANTS): (mass, energy) of every time level solved
    int log_inv = 0;
    double* inv_dev = nullptr;  // n_windows * nt pairs
    long long inv_count = 0;    // levels logged by the last solve
};

namespace pint {

template <class T> static Tabs<T>& tabs_of(pint_handle* h) { return *reinterpret_cast<Tabs<T>*>(h->tabs_ptrs); }

// Layout of the tables block (elements of T; complex = 2 T).
struct TabLayout {
    size_t twt, twx, twy, wx, wy, fx, ix, fy, iy, dsx, dsy, lamx, lamy, lam1, lam2, total;
};
static TabLayout tab_layout(const pint_problem* p, int fft_x, int fft_y) {
    TabLayout L{};
    const size_t nx = p->nx, ny = p->dim == 2 ? p->ny : 1, nt = p->nt;
    size_t o = 0;
    auto take = [&](size_t n) { size_t a = o; o += (n + 7) / 8 * 8; return a; };
    L.twt = take(2 * nt);
    L.twx = take(2 * nx);
    L.twy = take(2 * ny);
    L.wx = take(2 * nx);
    L.wy = take(2 * ny);
    L.fx = take(fft_x ? 0 : nx * nx);
    L.ix = take(fft_x ? 0 : nx * nx);
    const bool dy = p->dim == 2 && !fft_y;
    L.fy = take(dy ? ny * ny : 0);
    L.iy = take(dy ? ny * ny : 0);
    L.dsx = take(fft_x == 2 ? 4 * (nx + 1) : 0);
    L.dsy = take(p->dim == 2 && fft_y == 2 ? 4 * (ny + 1) : 0);
    L.lamx = take(nx);
    L.lamy = take(ny);
    L.lam1 = take(2 * (nt / 2 + 1));
    L.lam2 = take(2 * (nt / 2 + 1));
    L.total = o;
    return L;
}

// Dense basis of one axis: F[p][j] (forward) and Fi[j][p] (inverse).
static void dense_basis(int n, int bc, std::vector<double>& F, std::vector<double>& Fi) {
    F.assign((size_t)n * n, 0.0);
    Fi.assign((size_t)n * n, 0.0);
    for (int p = 0; p < n; ++p)
        for (int j = 0; j < n; ++j) {
            double f, fi;
            if (bc == PINT_BC_SIMPLY_SUPPORTED) {  // DST-I: sin(pi (p+1)(j+1)/(n+1)), inverse 2/(n+1) F^T
                f = sin(M_PI * (double)((long)(p + 1) * (j + 1) % (2 * (n + 1))) / (n + 1));
                fi = 2.0 / (n + 1) * f;
            } else if (bc == PINT_BC_NEUMANN_VERTEX) {
                // DCT-I: x_j = sum_p X_p cos(pi p j/(n-1)); X_p = 2/(n-1) c_p sum_j c_j x_j cos(...),
                // c = 1/2 at the two ends, 1 inside
                const double c = cos(M_PI * (double)(((long)p * j) % (2 * (n - 1))) / (n - 1));
                const double cp = (p == 0 || p == n - 1) ? 0.5 : 1.0, cj = (j == 0 || j == n - 1) ? 0.5 : 1.0;
                f = 2.0 / (n - 1) * cp * cj * c;
                fi = c;
            } else {  // DCT-II: cos(pi p (j+1/2)/n), inverse (1 or 2)/n F^T
                f = cos(M_PI * (double)(((long)p * (2 * j + 1)) % (4 * n)) / (2.0 * n));
                fi = (p == 0 ? 1.0 : 2.0) / n * f;
            }
            F[(size_t)p * n + j] = f;
            Fi[(size_t)j * n + p] = fi;
        }
}

template <class T>
static int build_tables(pint_handle* h) {
    const pint_problem* p = &h->p;
    const int nx = p->nx, ny = p->dim == 2 ? p->ny : 1, nt = p->nt;
    TabLayout L = tab_layout(p, h->fft_x, h->fft_y);
    std::vector<T> host(L.total, T(0));
    auto cset = [&](size_t off, int i, std::complex<double> z) {
        host[off + 2 * i] = (T)z.real();
        host[off + 2 * i + 1] = (T)z.imag();
    };
    auto expi = [](double turns) {  // exp(2 pi i * turns), turns a dyadic rational
        return std::complex<double>(cos(2.0 * M_PI * turns), sin(2.0 * M_PI * turns));
    };
    for (int j = 0; j < nt; ++j) cset(L.twt, j, expi(-(double)j / nt));
    for (int j = 0; j < nx; ++j) cset(L.twx, j, expi(-(double)j / nx));
    for (int j = 0; j < ny; ++j) cset(L.twy, j, expi(-(double)j / ny));
    for (int j = 0; j < nx; ++j) cset(L.wx, j, expi(-(double)j / (4.0 * nx)));
    for (int j = 0; j < ny; ++j) cset(L.wy, j, expi(-(double)j / (4.0 * ny)));
    std::vector<double> F, Fi;
    if (!h->fft_x) {
        dense_basis(nx, p->bc, F, Fi);
        for (size_t i = 0; i < F.size(); ++i) { host[L.fx + i] = (T)F[i]; host[L.ix + i] = (T)Fi[i]; }
    }
    if (p->dim == 2 && !h->fft_y) {
        dense_basis(ny, p->bc, F, Fi);
        for (size_t i = 0; i < F.size(); ++i) { host[L.fy + i] = (T)F[i]; host[L.iy + i] = (T)Fi[i]; }
    }
    if (h->fft_x == 2)
        for (int j = 0; j < 2 * (nx + 1); ++j) cset(L.dsx, j, expi(-(double)j / (2.0 * (nx + 1))));
    if (p->dim == 2 && h->fft_y == 2)
        for (int j = 0; j < 2 * (ny + 1); ++j) cset(L.dsy, j, expi(-(double)j / (2.0 * (ny + 1))));
    for (int i = 0; i < nx; ++i) host[L.lamx + i] = (T)lap_eig(i, nx, p->bc);
    for (int i = 0; i < ny; ++i) host[L.lamy + i] = p->dim == 2 ? (T)lap_eig(i, ny, p->bc) : T(0);
    // Lemma 2.1 with the forward transform exp(-2 pi i nk/nt):
    //   lambda_1k = (1 - alpha^{1/nt} e^{-2 pi i k/nt}) / dt,  lambda_2k = theta + (1-theta) alpha^{1/nt} e^{...}
    const double dt = h->geo.dt, a1 = pow(p->alpha, 1.0 / nt);
    for (int k = 0; k <= nt / 2; ++k) {
        std::complex<double> z = a1 * expi(-(double)k / nt);
        cset(L.lam1, k, (1.0 - z) / dt);
        cset(L.lam2, k, p->theta + (1.0 - p->theta) * z);
    }
    if (cudaMemcpyAsync(h->tab, host.data(), L.total * sizeof(T), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
        return PINT_ECUDA;
    Tabs<T>* tb = new (std::nothrow) Tabs<T>;
    if (!tb) return PINT_ENOMEM;
    const T* base = reinterpret_cast<const T*>(h->tab);
    tb->twt = reinterpret_cast<const c_t<T>*>(base + L.twt);
    tb->twx = reinterpret_cast<const c_t<T>*>(base + L.twx);
    tb->twy = reinterpret_cast<const c_t<T>*>(base + L.twy);
    tb->wx = reinterpret_cast<const c_t<T>*>(base + L.wx);
    tb->wy = reinterpret_cast<const c_t<T>*>(base + L.wy);
    tb->fx = base + L.fx;
    tb->ix = base + L.ix;
    tb->fy = base + L.fy;
    tb->iy = base + L.iy;
    tb->dsx = reinterpret_cast<const c_t<T>*>(base + L.dsx);
    tb->dsy = reinterpret_cast<const c_t<T>*>(base + L.dsy);
    tb->lamx = base + L.lamx;
    tb->lamy = base + L.lamy;
    tb->lam1 = reinterpret_cast<const c_t<T>*>(base + L.lam1);
    tb->lam2 = reinterpret_cast<const c_t<T>*>(base + L.lam2);
    tb->dte = p->equation == PINT_CAHN_HILLIARD_EYRE ? (T)h->geo.dt : T(0);
    h->tabs_ptrs = tb;
    // gamma tables (always FP64: the scaling and unscaling are FP64 steps)
    std::vector<double> g(nt), gi(nt);
    for (int n = 0; n < nt; ++n) {
        g[n] = pow(p->alpha, (double)n / nt);
        gi[n] = pow(p->alpha, -(double)n / nt) / nt;
    }
    if (cudaMemcpyAsync(h->gam, g.data(), nt * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess) return PINT_ECUDA;
    if (cudaMemcpyAsync(h->ginv, gi.data(), nt * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess) return PINT_ECUDA;
    if (h->gdt) {
        std::vector<double> gd(nt);
        std::vector<float> ig(nt);
        for (int n = 0; n < nt; ++n) { gd[n] = g[n] * h->geo.inv_dt; ig[n] = (float)(1.0 / g[n]); }
        if (cudaMemcpyAsync(h->gdt, gd.data(), nt * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
            cudaMemcpyAsync(h->igamf, ig.data(), nt * sizeof(float), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            return PINT_ECUDA;
    }
    if (h->gamf) {
        std::vector<float> gf(nt), gif(nt);
        for (int n = 0; n < nt; ++n) { gf[n] = (float)g[n]; gif[n] = (float)gi[n]; }
        if (cudaMemcpyAsync(h->gamf, gf.data(), nt * sizeof(float), cudaMemcpyHostToDevice, h->st) != cudaSuccess) return PINT_ECUDA;
        if (cudaMemcpyAsync(h->ginvf, gif.data(), nt * sizeof(float), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            return PINT_ECUDA;
    }
    return PINT_OK;
}

// Tables of the shorter segment lengths nt/2, nt/4, ... (down to 16) used by
// the adaptive window policy: FFT twiddles, lambda_1k, lambda_2k and the gamma
// scalings depend on the segment length; every other table is shared.
template <class T>
static int build_levels(pint_handle* h) {
    if (h->nlev > 1) return PINT_OK;
    const pint_problem* p = &h->p;
    const double dt = h->geo.dt;
    auto expi = [](double turns) { return std::complex<double>(cos(2.0 * M_PI * turns), sin(2.0 * M_PI * turns)); };
    const Tabs<T>* base = reinterpret_cast<const Tabs<T>*>(h->lev[0].tabs);
    for (int L = p->nt / 2; L >= 16 && h->nlev < 11; L /= 2) {
        auto& lv = h->lev[h->nlev];
        const size_t nk = L / 2 + 1;
        const size_t tbytes = (2 * L + 4 * nk) * sizeof(T);
        const size_t bytes = tbytes + 3 * L * sizeof(double) + 3 * L * sizeof(float) + 256;
        if (cudaMallocAsync(&lv.block, bytes, h->st) != cudaSuccess) { cudaGetLastError(); return PINT_ENOMEM; }
        h->bytes += (long long)bytes;
        std::vector<T> t(2 * L + 4 * nk);
        for (int j = 0; j < L; ++j) { auto z = expi(-(double)j / L); t[2 * j] = (T)z.real(); t[2 * j + 1] = (T)z.imag(); }
        const double a1 = pow(p->alpha, 1.0 / L);
        for (size_t k = 0; k < nk; ++k) {
            std::complex<double> z = a1 * expi(-(double)k / L);
            std::complex<double> l1 = (1.0 - z) / dt, l2 = p->theta + (1.0 - p->theta) * z;
            t[2 * L + 2 * k] = (T)l1.real();
            t[2 * L + 2 * k + 1] = (T)l1.imag();
            t[2 * L + 2 * nk + 2 * k] = (T)l2.real();
            t[2 * L + 2 * nk + 2 * k + 1] = (T)l2.imag();
        }
        std::vector<double> g(L), gi(L), gd(L);
        std::vector<float> gf(L), gif(L), ig(L);
        for (int n = 0; n < L; ++n) {
            g[n] = pow(p->alpha, (double)n / L);
            gi[n] = pow(p->alpha, -(double)n / L) / L;
            gf[n] = (float)g[n];
            gif[n] = (float)gi[n];
            gd[n] = g[n] * h->geo.inv_dt;
            ig[n] = (float)(1.0 / g[n]);
        }
        char* b = reinterpret_cast<char*>(lv.block);
        const size_t o_g = (tbytes + 15) / 16 * 16, o_gi = o_g + L * sizeof(double), o_gf = o_gi + L * sizeof(double),
                     o_gif = o_gf + L * sizeof(float), o_gd = (o_gif + L * sizeof(float) + 15) / 16 * 16,
                     o_ig = o_gd + L * sizeof(double);
        if (cudaMemcpyAsync(b, t.data(), tbytes, cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
            cudaMemcpyAsync(b + o_g, g.data(), L * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
            cudaMemcpyAsync(b + o_gi, gi.data(), L * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
            cudaMemcpyAsync(b + o_gf, gf.data(), L * sizeof(float), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
            cudaMemcpyAsync(b + o_gif, gif.data(), L * sizeof(float), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
            cudaMemcpyAsync(b + o_gd, gd.data(), L * sizeof(double), cudaMemcpyHostToDevice, h->st) != cudaSuccess ||
            cudaMemcpyAsync(b + o_ig, ig.data(), L * sizeof(float), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            return PINT_ECUDA;
        Tabs<T>* tb = new (std::nothrow) Tabs<T>(*base);
        if (!tb) return PINT_ENOMEM;
        const T* tt = reinterpret_cast<const T*>(b);
        tb->twt = reinterpret_cast<const c_t<T>*>(tt);
        tb->lam1 = reinterpret_cast<const c_t<T>*>(tt + 2 * L);
        tb->lam2 = reinterpret_cast<const c_t<T>*>(tt + 2 * L + 2 * nk);
        lv.nt = L;
        lv.tabs = tb;
        lv.gam = reinterpret_cast<double*>(b + o_g);
        lv.ginv = reinterpret_cast<double*>(b + o_gi);
        lv.gamf = reinterpret_cast<float*>(b + o_gf);
        lv.ginvf = reinterpret_cast<float*>(b + o_gif);
        lv.gdt = reinterpret_cast<double*>(b + o_gd);
        lv.igamf = reinterpret_cast<float*>(b + o_ig);
        h->nlev++;
    }
    return PINT_OK;
}

// Make level li (segment length lev[li].nt) the current time axis.
static void activate_level(pint_handle* h, int li) {
    const auto& lv = h->lev[li];
    h->geo.nt = lv.nt;
    h->gff.nt = lv.nt;
    h->tabs_ptrs = lv.tabs;
    h->gam = lv.gam;
    h->ginv = lv.ginv;
    h->gamf = lv.gamf;
    h->ginvf = lv.ginvf;
    h->gdt = lv.gdt;
    h->igamf = lv.igamf;
    h->gfx.nt = lv.nt;
}

static void derive(const pint_problem* p, pint_handle* h) {
    Geo& g = h->geo;
    g.nx = p->nx;
    g.ny = p->dim == 2 ? p->ny : 1;
    g.dim = p->dim;
    g.bc = p->bc;
    g.nt = p->nt;
    g.nspace = g.nx * g.ny;
    g.dt = p->T / ((double)p->nt * p->n_windows);
    g.inv_dt = 1.0 / g.dt;
    const double hx = grid_h(p->nx, p->bc), hy = grid_h(g.ny, p->bc);
    g.ihx2 = 1.0 / (hx * hx);
    g.ihy2 = p->dim == 2 ? 1.0 / (hy * hy) : 0.0;
    h->coef.ch = 0;
    switch (p->equation) {
        case PINT_BIHARMONIC: g.c2 = 1.0; g.c1 = 0.0; g.cN = 0.0; break;
        case PINT_LINEAR_CH: g.c2 = p->eps * p->eps; g.c1 = p->beta * fabs(p->beta); g.cN = 0.0; break;   // signed beta^2
        default: g.c2 = p->eps * p->eps; g.c1 = 1.0; g.cN = -1.0; h->coef.ch = 1; break;
    }
    g.th = p->theta;
    g.expl = p->equation == PINT_CAHN_HILLIARD_EYRE ? 1 : 0;
    h->coef.c2 = g.c2;
    h->coef.c1 = g.expl ? 0.0 : g.c1;   // Eyre: the Laplacian term is explicit (lambda_3k in Step 2)
    h->fft_x = axis_fft(p->nx, p->bc, 4096);
    h->fft_y = p->dim == 2 ? axis_fft(g.ny, p->bc, 1024) : 1;
    GeoFF& f = h->gff;
    f.nx = g.nx;
    f.ny = g.ny;
    f.dim = g.dim;
    f.bc = g.bc;
    f.nt = g.nt;
    f.nspace = g.nspace;
    f.ihx2 = ff_from_double(g.ihx2);
    f.ihy2 = ff_from_double(g.ihy2);
    f.inv_dt = ff_from_double(g.inv_dt);
    const bool sq = g.dim == 1 || g.ihx2 == g.ihy2;   // must match launch_residual_ff
    // the float-float residual is evaluated scaled by dt: coefficients carry dt,
    // and theta (exact: 1 or 1/2), so that dt r = u_{n-1} - u_n - A'(u_n) - A'(u_{n-1})
    // with A' = theta dt A when theta = 1/2
    const double s2 = sq ? g.ihx2 * g.ihx2 : 1.0, s1 = sq ? g.ihx2 : 1.0;
    f.c2 = ff_from_double(g.c2 * s2 * g.dt * g.th);
    f.c1 = ff_from_double(g.c1 * s1 * g.dt * g.th);
    f.cN = ff_from_double(g.cN * s1 * g.dt * g.th);
    f.half = g.th < 1.0 ? 1 : 0;
    f.expl = g.expl;
    // stiffness dt * max |spectrum of the spatial operator|: above 1e7 the stencil
    // sums use chained accurate double-word additions (see k_residual_ff.cu)
    const double lam_max = 4.0 * g.ihx2 + (g.dim == 2 ? 4.0 * g.ihy2 : 0.0);
    const double mu_max = g.c2 * lam_max * lam_max + (fabs(g.c1) + 2.0 * fabs(g.cN)) * lam_max;
    f.accurate = g.dt * mu_max > 1e7 ? 1 : 0;
    h->gfx = make_geo_fx(g);
}

static Sizes sizes_of(const pint_problem* p, pint_handle* tmp) {
    derive(p, tmp);
    Sizes z{};
    z.nspace = (size_t)tmp->geo.nspace;
    z.dof = z.nspace * p->nt;
    z.nk = p->nt / 2 + 1;
    int gx, gy, gz, chunk;
    const int nres = residual_grid(tmp->geo, gx, gy, gz, chunk);
    const int nff = residual_ff_grid(tmp->geo, gx, gy, gz, chunk);
    const int nfx = residual_fx_grid(tmp->geo, gx, gy, gz, chunk);
    const int nn = norm2_blocks((int)z.nspace);
    z.partials = (size_t)std::max(std::max(nres, nfx), std::max(nff, nn));
    TabLayout L = tab_layout(p, tmp->fft_x, tmp->fft_y);
    z.tables_T = L.total;
    const size_t ts = f32_transforms(p) ? 4 : 8;
    z.tables_bytes = L.total * ts;
    return z;
}

static long long footprint_of(const pint_problem* p) {
    pint_handle tmp;
    memset(&tmp.p, 0, sizeof(tmp.p));
    Sizes z = sizes_of(p, &tmp);
    const size_t ts = f32_transforms(p) ? 4 : 8;
    long long b = 0;
    b += sizeof(Ctl);
    b += z.partials * 2 * sizeof(double);
    b += std::max<size_t>(z.nspace / 16 + 2, (size_t)time_inv_blocks(p->nt, (int)z.nspace, f32_transforms(p))) * 2 *
         sizeof(double);
    b += 2 * (size_t)p->nt * sizeof(double);
    b += z.nspace * sizeof(double) * (needs_b1(p) ? 2 : 1);
    b += z.dof * ts;                 // s
    b += z.nk * z.nspace * 2 * ts;   // S
    b += z.tables_bytes;
    if (p->precision == PINT_MIXED_FF) b += z.dof * 8 + z.nspace * 8 + 2 * (size_t)p->nt * 4;
    if (p->precision == PINT_MIXED) b += (size_t)p->nt * (sizeof(double) + sizeof(float));
    if (f32_transforms(p) && time_gemm_supported(p->nt, (int)z.nspace)) b += (size_t)4 * p->nt * p->nt * 2;
    return b;
}

// Step 2 as one fused kernel per iteration (square 2-D grids up to 256^2).
static bool fused_spatial(const pint_handle* h) {
    return h->fuse2d && slice2d_supported(h->geo, h->fft_x, h->fft_y, h->p.precision != PINT_FP64);
}
// 1-D long time axes on the cosine path: Step 2 rides on the pack of the
// inverse time transform (not with the space-varying Jacobian, whose inner
// solve works on the half spectrum itself).
static bool long_fused(const pint_handle* h) {
    return h->geo.dim == 1 && h->geo.nt > 1024 && h->fft_x == 1 && !(h->vary > 0 && h->coef.ch);
}
static int spatial_launches(const pint_handle* h) {
    return long_fused(h) ? 0 : fused_spatial(h) ? 1 : (h->geo.dim == 2 ? 3 : 1);
}

// Partial-sum buffer of the update-size test, or NULL when the test is off
// (then the inverse time transform skips that reduction).
static double* upd_part(pint_handle* h) { return h->p.tol_update > 0.0 ? h->dpart : nullptr; }

// ---------------------------------------------------------------------------
// Phase accounting
// ---------------------------------------------------------------------------
enum { PH_RES = 0, PH_CHECK = 1, PH_TFWD = 2, PH_SP0 = 3, PH_SP1 = 4, PH_SP2 = 5, PH_TINV = 6, PH_SETUP = 7 };

static void prof_flush(pint_handle* h) {  // stream must be idle past the recorded events
    for (int i = 0; i < h->nev; ++i) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess) h->ms[h->ev_phase[i]] += t;
        else cudaGetLastError();
    }
    h->nev = 0;
}
// prof_on 2 (coarse): events only around the residual with its check (booked
// to PH_RES) and around the whole diagonalized step, Steps 1-3 (booked to
// PH_TFWD), so that the event records do not split the step's kernels.
static bool prof_coarse_skip_begin(const pint_handle* h, int ph) {
    return h->prof_on == 2 && ph != PH_RES && ph != PH_TFWD && ph != PH_SETUP;
}
static bool prof_coarse_skip_end(const pint_handle* h, int ph) {
    return h->prof_on == 2 && ph != PH_CHECK && ph != PH_TINV && ph != PH_SETUP;
}
static void prof_begin(pint_handle* h, int ph) {
    if (!h->prof_on || prof_coarse_skip_begin(h, ph)) return;
    if (h->nev == pint_handle::NEV) {
        cudaStreamSynchronize(h->st);
        prof_flush(h);
    }
    h->ev_phase[h->nev] = ph;
    cudaEventRecord(h->ev[2 * h->nev], h->st);
}
static void prof_end(pint_handle* h, int ph, int nlaunch) {
    h->launches[ph] += nlaunch;
    if (!h->prof_on || prof_coarse_skip_end(h, ph)) return;
    cudaEventRecord(h->ev[2 * h->nev + 1], h->st);
    h->nev++;
}

// ---------------------------------------------------------------------------
// The iteration
// ---------------------------------------------------------------------------
// Whether the tensor-core transforms apply to the current time axis (the table
// is built for the handle's N_t; shorter adaptive segments use the FFT).
static bool gemm_ok(const pint_handle* h) {
    return h->wgemm && h->geo.nt == h->p.nt && time_gemm_supported(h->geo.nt, h->geo.nspace);
}
static bool use_gemm_fwd(const pint_handle* h) { return h->gemm_fwd && gemm_ok(h); }
static bool use_gemm_inv(const pint_handle* h) {
    return h->gemm_inv && gemm_ok(h) && h->p.precision == PINT_MIXED;
}
// Step 1 on the FP32 path: DFT matrix product or FFT
static cudaError_t tfwd_f32(pint_handle* h, const float* s, float2* S) {
    const Geo& g = h->geo;
    if (use_gemm_fwd(h)) return launch_time_gemm(0, g.nt, g.nspace, s, S, h->wgemm, nullptr, h->ctl, nullptr, h->st);
    return launch_time_fwd<float>(g.nt, g.nspace, s, S, tabs_of<float>(h).twt, h->ctl, h->st);
}
// CTAs writing update-size partials in Step 3 of PINT_MIXED
static int tinv_blocks(pint_handle* h) {
    return use_gemm_inv(h) ? time_gemm_blocks(h->geo.nspace) : time_inv_blocks(h->geo.nt, h->geo.nspace, 1);
}

template <class T> struct Impl {
    // Step 2's scalar-Jacobian divide of every frequency slice; the kernels read
    // status and jbar from ctl (the handle's control word unless given).
    static cudaError_t spatial(pint_handle* h, c_t<T>* S, const Tabs<T>& tb, const Ctl* ctl = nullptr) {
        if (!ctl) ctl = h->ctl;
        if (fused_spatial(h)) {
            prof_begin(h, PH_SP0);
            cudaError_t e = launch_slice2d<T>(h->geo, S, tb, h->coef, ctl, h->st);
            prof_end(h, PH_SP0, 1);
            return e;
        }
        const int nst = h->geo.dim == 2 ? 3 : 1;
        for (int stg = 0; stg < nst; ++stg) {
            prof_begin(h, PH_SP0 + stg);
            cudaError_t e = launch_spatial_stage<T>(stg, h->geo, S, tb, h->coef, h->fft_x, h->fft_y, ctl, h->st);
            prof_end(h, PH_SP0 + stg, 1);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    // Step 2 with the space-varying Jacobian J~(x) (Eq. 4.12): one cycle of
    // flexible GMRES on the block-diagonal system M_k x_k = S1_k over all
    // frequencies at once, right-preconditioned by the scalar-J-bar divide,
    // started from that divide's result.  Complex dot products: per-thread sums
    // in the vectors' precision, CTA and grid sums in FP64.  The cycle runs
    // entirely on the device: one-CTA kernels add the dot products' partials in
    // a fixed order and keep the Hessenberg matrix, the rotations and the stop
    // test (GmState); the launch sequence is the same for every cycle (vector
    // kernels skip once the cycle has stopped), so it can be captured.
    static cudaError_t step2_varying(pint_handle* h, c_t<T>* S, const Tabs<T>& tb, const double* U, const float2* uff) {
        using C = c_t<T>;
        const Geo& g = h->geo;
        const int nk = g.nt / 2 + 1, m = h->vary;
        const size_t ns = (size_t)g.nspace, n = (size_t)nk * ns;
        const int nbx = cdot_blocks(ns, nk);
        C* X = reinterpret_cast<C*>(h->jbuf);   // the right-hand side S1 stays in S until the end
        C* V = X + n;
        C* Z = V + (size_t)(m + 1) * n;
        T* jt = reinterpret_cast<T*>(h->jt);
        GmHead* gh = h->gmh;
        GmK* gk = h->gmk;
        const int* skip = &gh->skip;
        double* part2 = h->jpart + 2 * (size_t)nbx * nk;
        const double c1 = g.expl ? 0.0 : 1.0;
        cudaError_t e;
        launch_jtilde<T>(U, uff, g.nt, g.nspace, jt, h->st);
        launch_gm_reset(gh, h->st);
        launch_caxpby<T>(X, 1.0, S, 0.0, nullptr, n, nullptr, nullptr, h->st);
        if ((e = spatial(h, X, tb)) != cudaSuccess) return e;           // x0 = P^{-1} S1
        launch_apply_M<T>(g, nk, X, V, jt, tb, h->coef.c2, c1, nullptr, S, h->st);   // r0 = S1 - M x0
        launch_cmulti_dot<T>(S, S, n, 1, ns, nk, h->jpart, nullptr, h->st);
        launch_cmulti_dot<T>(V, V, n, 1, ns, nk, part2, nullptr, h->st);
        launch_gm_init(h->jpart, part2, nbx, h->ctl, gh, gk, nk, h->vary_tol, h->st);
        launch_cmulti_axpy<T>(V, V, n, 0, 0, ns, nk, gk, GM_COEF, skip, h->st, nullptr, 1);   // v_0 = r0 / ||r0||
        for (int j = 0; j < m; ++j) {
            C* vj = V + (size_t)j * n;
            C* zj = Z + (size_t)j * n;
            C* w = V + (size_t)(j + 1) * n;
            launch_caxpby<T>(zj, 1.0, vj, 0.0, nullptr, n, skip, nullptr, h->st);
            if ((e = spatial(h, zj, tb, &gh->ictl)) != cudaSuccess) return e;   // z_j = P^{-1} v_j
            launch_apply_M<T>(g, nk, zj, w, jt, tb, h->coef.c2, c1, skip, nullptr, h->st);
            // classical Gram-Schmidt per slice: <v_i, w> for i <= j and <w, w> in one pass (w is v_{j+1});
            // a second pass for the slices whose ||w - sum h_i v_i||^2 = <w, w> - sum |h_i|^2 cancels
            launch_cmulti_dot<T>(w, V, n, j + 2, ns, nk, h->jpart, skip, h->st);
            launch_gm_orth1(h->jpart, nbx, j, gh, gk, nk, h->st);
            launch_cmulti_axpy<T>(w, V, n, j + 1, j + 1, ns, nk, gk, GM_COEFA, &gh->skip_re[j], h->st);
            launch_cmulti_dot<T>(w, V, n, j + 2, ns, nk, h->jpart, &gh->skip_re[j], h->st);
            launch_gm_orth2(h->jpart, nbx, j, gh, gk, nk, h->vary_tol, h->st);
            // v_{j+1} = (w - sum h_i v_i) / h_{j+1,j}
            launch_cmulti_axpy<T>(w, V, n, j + 1, j + 1, ns, nk, gk, GM_COEF, skip, h->st, nullptr, 1);
        }
        launch_gm_solve(gk, nk, h->st);
        // S2 = x0 + Z y over the steps run (z_i beyond them were never written)
        launch_cmulti_axpy<T>(X, Z, n, m, m, ns, nk, gk, GM_Y, nullptr, h->st, S, 0, &gh->jmax);
        return cudaGetLastError();
    }
    static cudaError_t step2(pint_handle* h, c_t<T>* S, const Tabs<T>& tb, const double* U, const float2* uff) {
        if (h->vary > 0 && h->coef.ch) return step2_varying(h, S, tb, U, uff);
        return spatial(h, S, tb);
    }
    static cudaError_t iteration(pint_handle* h, double* U, const double* u0w) {
        const Geo& g = h->geo;
        T* s = reinterpret_cast<T*>(h->s);
        c_t<T>* S = reinterpret_cast<c_t<T>*>(h->S);
        const Tabs<T>& tb = tabs_of<T>(h);
        prof_begin(h, PH_RES);
        int gx, gy, gz, chunk, np;
        if (std::is_same<T, float>::value && h->use_fx) {
            // FP64-accurate residual and alpha-scaling in block fixed point (integer pipes)
            cudaError_t e = launch_residual_fx(h->gfx, g, U, u0w, h->gdt, h->igamf, reinterpret_cast<float*>(s),
                                               nullptr, h->partials, h->ctl, h->st, 0);
            if (e != cudaSuccess) return e;
            np = residual_fx_grid(g, gx, gy, gz, chunk);
        } else {
            launch_residual<T>(g, U, u0w, h->gam, nullptr, s, h->partials, h->ctl, h->st);
            np = residual_grid(g, gx, gy, gz, chunk);
        }
        prof_end(h, PH_RES, 1);
        prof_begin(h, PH_CHECK);
        const int ndp = !upd_part(h) ? 0 : std::is_same<T, float>::value ? tinv_blocks(h)
                                                                          : time_inv_blocks(g.nt, g.nspace, 0);
        launch_after_residual(h->partials, np, 1.0 / ((double)g.nt * g.nspace), h->ctl, h->st, h->gcond, h->capturing,
                              upd_part(h), ndp);
        prof_end(h, PH_CHECK, 1);
        prof_begin(h, PH_TFWD);
        cudaError_t e;
        if constexpr (std::is_same<T, float>::value) {
            e = tfwd_f32(h, s, S);
            prof_end(h, PH_TFWD, use_gemm_fwd(h) ? 1 : time_fwd_launches(g.nt));
        } else {
            e = launch_time_fwd<T>(g.nt, g.nspace, s, S, tb.twt, h->ctl, h->st);
            prof_end(h, PH_TFWD, time_fwd_launches(g.nt));
        }
        if (e != cudaSuccess) return e;
        const bool lf = long_fused(h);
        const LongSolve<T> ls{&tb, h->coef, g.nx};
        if (!lf && (e = step2(h, S, tb, U, nullptr)) != cudaSuccess) return e;
        prof_begin(h, PH_TINV);
        if (std::is_same<T, float>::value && use_gemm_inv(h)) {
            e = launch_time_gemm(1, g.nt, g.nspace, S, U, h->wgemm, h->ginv, h->ctl, upd_part(h), h->st);
            prof_end(h, PH_TINV, 1);
        } else {
            e = launch_time_inv<T>(g.nt, g.nspace, S, tb.twt, h->ginv, U, 1, h->ctl, upd_part(h), h->st, h->s,
                                   lf ? &ls : nullptr);
            prof_end(h, PH_TINV, time_inv_launches(g.nt));
        }
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    static cudaError_t precond(pint_handle* h, double jbar, const double* r, double* delta) {
        const Geo& g = h->geo;
        T* s = reinterpret_cast<T*>(h->s);
        c_t<T>* S = reinterpret_cast<c_t<T>*>(h->S);
        const Tabs<T>& tb = tabs_of<T>(h);
        launch_set_running(h->ctl, jbar, h->st);
        launch_scale_cast<T>(r, h->gam, s, g.nspace, g.nt, h->st);
        cudaError_t e;
        if constexpr (std::is_same<T, float>::value) e = tfwd_f32(h, s, S);
        else e = launch_time_fwd<T>(g.nt, g.nspace, s, S, tb.twt, h->ctl, h->st);
        if (e != cudaSuccess) return e;
        const bool lf = long_fused(h);
        const LongSolve<T> ls{&tb, h->coef, g.nx};
        if (!lf && (e = spatial(h, S, tb)) != cudaSuccess) return e;
        if (std::is_same<T, float>::value && use_gemm_inv(h)) {
            // the matrix-product inverse accumulates: delta = 0 + P^{-1} r
            if ((e = cudaMemsetAsync(delta, 0, (size_t)g.nt * g.nspace * sizeof(double), h->st)) != cudaSuccess) return e;
            e = launch_time_gemm(1, g.nt, g.nspace, S, delta, h->wgemm, h->ginv, h->ctl, nullptr, h->st);
        } else {
            e = launch_time_inv<T>(g.nt, g.nspace, S, tb.twt, h->ginv, delta, 0, h->ctl, nullptr, h->st, h->s,
                                   lf ? &ls : nullptr);
        }
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
};

// Iteration k = 0 from the zero iterate: r_0 = b is known, so the residual
// and the forward time transform are replaced by writing the spectrum of b.
static cudaError_t zero_start(pint_handle* h, double* U, const double* u0w) {
    const Geo& g = h->geo;
    const int nk = g.nt / 2 + 1;
    prof_begin(h, PH_TFWD);
    // spectrum of b: b_1 at every frequency (theta = 1: b_1 = u0/dt; else computed at the window start)
    const bool nb = g.th < 1.0 || g.expl;
    const double* b1 = nb ? h->b1 : u0w;
    const double sc = nb ? 1.0 : g.inv_dt;
    if (f32_transforms(&h->p)) launch_zero_start<float>(reinterpret_cast<float2*>(h->S), b1, sc, g.nspace, nk, h->ctl, h->st);
    else launch_zero_start<double>(reinterpret_cast<double2*>(h->S), b1, sc, g.nspace, nk, h->ctl, h->st);
    prof_end(h, PH_TFWD, 1);
    cudaError_t e;
    const bool lf = long_fused(h);
    if (f32_transforms(&h->p)) {
        const Tabs<float>& tb = tabs_of<float>(h);
        const LongSolve<float> ls{&tb, h->coef, g.nx};
        if (!lf && (e = Impl<float>::spatial(h, reinterpret_cast<float2*>(h->S), tb)) != cudaSuccess) return e;
        prof_begin(h, PH_TINV);
        if (h->p.precision == PINT_MIXED_FF)
            e = launch_time_inv_ff(g.nt, g.nspace, reinterpret_cast<float2*>(h->S), tb.twt, h->ginvf, h->Uff_cur, h->ctl,
                                   upd_part(h), h->st, h->s, lf ? &ls : nullptr);
        else if (use_gemm_inv(h))
            e = launch_time_gemm(1, g.nt, g.nspace, h->S, U, h->wgemm, h->ginv, h->ctl, upd_part(h), h->st);
        else
            e = launch_time_inv<float>(g.nt, g.nspace, reinterpret_cast<float2*>(h->S), tb.twt, h->ginv, U, 1, h->ctl,
                                       upd_part(h), h->st, h->s, lf ? &ls : nullptr);
        prof_end(h, PH_TINV, (h->p.precision != PINT_MIXED_FF && use_gemm_inv(h)) ? 1 : time_inv_launches(g.nt));
    } else {
        const Tabs<double>& tb = tabs_of<double>(h);
        const LongSolve<double> ls{&tb, h->coef, g.nx};
        if (!lf && (e = Impl<double>::spatial(h, reinterpret_cast<double2*>(h->S), tb)) != cudaSuccess) return e;
        prof_begin(h, PH_TINV);
        e = launch_time_inv<double>(g.nt, g.nspace, reinterpret_cast<double2*>(h->S), tb.twt, h->ginv, U, 1, h->ctl,
                                    upd_part(h), h->st, h->s, lf ? &ls : nullptr);
        prof_end(h, PH_TINV, time_inv_launches(g.nt));
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// PINT_MIXED_FF: float-float residual and update, FP32 transforms.
static cudaError_t iteration_ff(pint_handle* h) {
    const Geo& g = h->geo;
    float* s = reinterpret_cast<float*>(h->s);
    float2* S = reinterpret_cast<float2*>(h->S);
    const Tabs<float>& tb = tabs_of<float>(h);
    prof_begin(h, PH_RES);
    launch_residual_ff(h->gff, g, h->Uff_cur, h->u0ff, h->gamf, s, h->partials, h->ctl, h->st);
    prof_end(h, PH_RES, 1);
    int gx, gy, gz, chunk;
    const int np = residual_ff_grid(g, gx, gy, gz, chunk);
    prof_begin(h, PH_CHECK);
    launch_after_residual(h->partials, np, 1.0 / ((double)g.nt * g.nspace), h->ctl, h->st, h->gcond, h->capturing,
                              upd_part(h), upd_part(h) ? time_inv_ff_blocks(g.nt, g.nspace, h->ctl) : 0);
    prof_end(h, PH_CHECK, 1);
    prof_begin(h, PH_TFWD);
    cudaError_t e = tfwd_f32(h, s, S);
    prof_end(h, PH_TFWD, use_gemm_fwd(h) ? 1 : time_fwd_launches(g.nt));
    if (e != cudaSuccess) return e;
    const bool lf = long_fused(h);
    const LongSolve<float> ls{&tb, h->coef, g.nx};
    if (!lf && (e = Impl<float>::step2(h, S, tb, nullptr, h->Uff_cur)) != cudaSuccess) return e;
    prof_begin(h, PH_TINV);
    e = launch_time_inv_ff(g.nt, g.nspace, S, tb.twt, h->ginvf, h->Uff_cur, h->ctl, upd_part(h), h->st, h->s,
                           lf ? &ls : nullptr);
    prof_end(h, PH_TINV, time_inv_launches(g.nt));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

static cudaError_t iteration(pint_handle* h, double* U, const double* u0w) {
    return f32_transforms(&h->p) ? Impl<float>::iteration(h, U, u0w) : Impl<double>::iteration(h, U, u0w);
}


// The iteration loop of one window as a CUDA graph: a while-node whose body is
// one iteration (residual, check, time FFT, spatial stages, inverse FFT); the
// check kernel sets the loop condition from the device status word, so the
// whole solve of a window is one graph launch with no host round trip.  The
// body of PINT_MIXED_FF touches handle-owned buffers only; the other modes
// also bake U and the window's u0 in, so graphs are cached per (U, u0).
static cudaGraphExec_t get_graph(pint_handle* h, double* U, const double* u0w) {
    const bool ffm = h->p.precision == PINT_MIXED_FF;
    const void* kU = ffm ? (const void*)h->Uff_cur : U;
    const void* ku0 = ffm ? nullptr : u0w;
    for (auto& sl : h->gslot)
        if (sl.exec && sl.U == kU && sl.u0 == ku0) return sl.exec;
    if (!h->capst && cudaStreamCreateWithFlags(&h->capst, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) return nullptr;
    bool ok = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    ok = ok && cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaStream_t saved = h->st;
        const int prof = h->prof_on;
        h->st = h->capst;
        h->prof_on = 0;
        h->capturing = 1;
        h->gcond = (unsigned long long)cond;
        long long saved_launches[PINT_NPHASE];
        memcpy(saved_launches, h->launches, sizeof(saved_launches));
        ok = cudaStreamBeginCaptureToGraph(h->capst, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
             cudaSuccess;
        if (ok) {
            cudaError_t e = ffm ? iteration_ff(h) : iteration(h, U, u0w);
            cudaGraph_t outg = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(h->capst, &outg);
            ok = e == cudaSuccess && e2 == cudaSuccess;
        }
        memcpy(h->launches, saved_launches, sizeof(saved_launches));
        h->st = saved;
        h->prof_on = prof;
        h->capturing = 0;
        h->gcond = 0;
    }
    ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        return nullptr;
    }
    auto& sl = h->gslot[h->gnext];
    h->gnext ^= 1;
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
    sl.exec = exec;
    sl.U = kU;
    sl.u0 = ku0;
    sl.cond = (unsigned long long)cond;
    return exec;
}

// Validation and geometry for callers without a handle (pint_residual_static).
int validate_problem(const pint_problem* p) { return validate(p); }

void geometry_of(const pint_problem* p, Geo& g) {
    g.nx = p->nx;
    g.ny = p->dim == 2 ? p->ny : 1;
    g.dim = p->dim;
    g.bc = p->bc;
    g.nt = p->nt;
    g.nspace = g.nx * g.ny;
    g.dt = p->T / ((double)p->nt * p->n_windows);
    g.inv_dt = 1.0 / g.dt;
    const double hx = grid_h(p->nx, p->bc), hy = grid_h(g.ny, p->bc);
    g.ihx2 = 1.0 / (hx * hx);
    g.ihy2 = p->dim == 2 ? 1.0 / (hy * hy) : 0.0;
    switch (p->equation) {
        case PINT_BIHARMONIC: g.c2 = 1.0; g.c1 = 0.0; g.cN = 0.0; break;
        case PINT_LINEAR_CH: g.c2 = p->eps * p->eps; g.c1 = p->beta * fabs(p->beta); g.cN = 0.0; break;   // signed beta^2
        default: g.c2 = p->eps * p->eps; g.c1 = 1.0; g.cN = -1.0; break;
    }
    g.th = p->theta;
    g.expl = p->equation == PINT_CAHN_HILLIARD_EYRE ? 1 : 0;
}

// dt * max|spectrum| of the spatial operator (for Cahn-Hilliard with the
// linear part's coefficient |1 - jbar| bounded by 1 + 2 * 3 u^2 at |u| <= 1).
double stiffness_of(const pint_problem* p) {
    Geo g;
    geometry_of(p, g);
    const double lam_max = 4.0 * g.ihx2 + (g.dim == 2 ? 4.0 * g.ihy2 : 0.0);
    const double mu_max = g.c2 * lam_max * lam_max + (fabs(g.c1) + 2.0 * fabs(g.cN)) * lam_max;
    return g.dt * mu_max;
}

// Precision a problem runs in.  The FP32 inner solves act as a preconditioner
// refined by the outer iteration, which needs their error amplified by the
// stiff operator, amp = 2^-24 dt max|spectrum|, to stay small:
//  * linear equations: as requested up to amp 1; up to amp 1e3 with an FP64
//    residual and iterate (PINT_MIXED: the float-float iterate's own rounding
//    floor, 2^-49 dt max|spectrum|, would then stall the stop tests); beyond,
//    FP64 throughout (the FP32 rounding of the correction's high modes then
//    dominates the next residual: observed residual growth of 1e7 on a 1-D
//    biharmonic of 4096 cells at amp 8e4);
//  * Cahn-Hilliard, whose Jacobian moves between iterations: as requested up to
//    amp 0.1, FP64 beyond (observed divergence of 1-D instances at 0.87); 2-D
//    PinT-I in PINT_MIXED up to amp 0.5 (its FP64-accurate residual runs on the
//    integer pipes; measured convergence on every such instance of the batched
//    and served pools).
int effective_precision(const pint_problem* p) {
    if (p->precision == PINT_FP64) return PINT_FP64;
    const double amp = stiffness_of(p) * 0x1p-24;
    if (p->equation == PINT_CAHN_HILLIARD || p->equation == PINT_CAHN_HILLIARD_EYRE) {
        // 2-D PinT-I in PINT_MIXED (its residual in block fixed point) is refined up to amp 0.5
        const bool wide = p->precision == PINT_MIXED && p->equation == PINT_CAHN_HILLIARD && p->dim == 2;
        return amp > (wide ? 0.5 : 0.1) ? PINT_FP64 : p->precision;
    }
    if (amp <= 1.0) return p->precision;
    return amp <= 1e3 ? PINT_MIXED : PINT_FP64;
}

}  // namespace pint

using namespace pint;

#define PINT_CK(call)                                  \
    do {                                               \
        if ((call) != cudaSuccess) return PINT_ECUDA;  \
    } while (0)

extern "C" {

const char* pint_strerror(int code) {
    switch (code) {
        case PINT_OK: return "ok";
        case PINT_EINVAL: return "invalid or unsupported parameter";
        case PINT_ENOMEM: return "out of memory";
        case PINT_ECUDA: return "CUDA runtime error";
        case PINT_ENOCONV: return "iteration did not reach the tolerance within max_iter";
        case PINT_EDIVERGED: return "iteration diverged (residual non-finite or grew by 1e6)";
        default: return "unknown pint error code";
    }
}

long long pint_footprint(const pint_problem* p) {
    int rc = validate(p);
    if (rc != PINT_OK) return rc;
    pint_problem q = *p;
    q.precision = effective_precision(p);
    return footprint_of(&q);
}

void pint_destroy(pint_handle* h) {
    if (!h) return;
    // stream-ordered frees: destroying a handle does not wait for the whole device
    cudaStream_t fs = h->st;
    auto af = [&](void* q) { if (q) cudaFreeAsync(q, fs); };
    af(h->ctl);
    ctl_slab_release(h->hctl);
    af(h->partials);
    af(h->dpart);
    af(h->kv);
    af(h->kz);
    af(h->kzero);
    af(h->kpart);
    af(h->kcoef);
    af(h->jbuf);
    af(h->jt);
    af(h->jpart);
    af(h->gmh);
    af(h->gmk);
    af(h->inv_dev);
    af(h->wgemm);
    if (h->nlev > 0) activate_level(h, 0);   // the base level owns gam/ginv/gamf/ginvf and tabs_ptrs
    for (int i = 1; i < h->nlev; ++i) {
        af(h->lev[i].block);
        if (f32_transforms(&h->p)) delete reinterpret_cast<Tabs<float>*>(h->lev[i].tabs);
        else delete reinterpret_cast<Tabs<double>*>(h->lev[i].tabs);
    }
    af(h->gam);
    af(h->ginv);
    af(h->gdt);
    af(h->igamf);
    af(h->u0buf);
    af(h->b1);
    af(h->hU);
    af(h->hu0);
    af(h->s);
    af(h->S);
    af(h->tab);
    af(h->Uff);
    af(h->u0ff);
    af(h->gamf);
    af(h->ginvf);
    for (int i = 0; i < 2 * pint_handle::NEV; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    for (auto& sl : h->gslot)
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (h->capst) cudaStreamDestroy(h->capst);
    if (h->tabs_ptrs) {
        if (f32_transforms(&h->p)) delete reinterpret_cast<Tabs<float>*>(h->tabs_ptrs);
        else delete reinterpret_cast<Tabs<double>*>(h->tabs_ptrs);
    }
    delete h;
}

int pint_create(const pint_problem* p, void* cuda_stream, pint_handle** out) {
    if (!out) return PINT_EINVAL;
    *out = nullptr;
    int rc = validate(p);
    if (rc != PINT_OK) return rc;
    pint_problem q = *p;
    q.precision = effective_precision(p);
    p = &q;
    if (configure_kernels() != cudaSuccess) return PINT_ECUDA;
    pint_handle* h = new (std::nothrow) pint_handle;
    if (!h) return PINT_ENOMEM;
    h->p = *p;
    h->st = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return PINT_ECUDA;
    }
    Sizes z = sizes_of(p, h);   // also derives the geometry and the axis paths
    if ((h->fft_x == 2 && configure_dst(p->nx, 0, f32_transforms(p)) != cudaSuccess) ||
        (p->dim == 2 && h->fft_y == 2 && configure_dst(p->ny, 1, f32_transforms(p)) != cudaSuccess)) {
        delete h;
        return PINT_ECUDA;
    }
    const size_t ts = f32_transforms(p) ? 4 : 8;
    auto dalloc = [&](void** ptr, size_t bytes) -> int {
        if (cudaMallocAsync(ptr, bytes < 16 ? 16 : bytes, h->st) != cudaSuccess) {
            cudaGetLastError();
            return PINT_ENOMEM;
        }
        h->bytes += (long long)bytes;
        return PINT_OK;
    };
    rc = PINT_OK;
    if (!rc) rc = dalloc((void**)&h->ctl, sizeof(Ctl));
    if (!rc) rc = dalloc((void**)&h->partials, z.partials * 2 * sizeof(double));
    const size_t ndp = std::max<size_t>(z.nspace / 16 + 2, (size_t)time_inv_blocks(p->nt, (int)z.nspace, f32_transforms(p)));
    if (!rc) rc = dalloc((void**)&h->dpart, ndp * 2 * sizeof(double));
    if (!rc) rc = dalloc((void**)&h->gam, p->nt * sizeof(double));
    if (!rc) rc = dalloc((void**)&h->ginv, p->nt * sizeof(double));
    if (!rc) rc = dalloc((void**)&h->u0buf, z.nspace * sizeof(double));
    if (!rc && needs_b1(p)) rc = dalloc((void**)&h->b1, z.nspace * sizeof(double));
    if (!rc) rc = dalloc(&h->s, z.dof * ts);
    if (!rc) rc = dalloc(&h->S, z.nk * z.nspace * 2 * ts);
    if (!rc) rc = dalloc(&h->tab, z.tables_bytes);
    if (!rc && p->precision == PINT_MIXED) {
        rc = dalloc((void**)&h->gdt, p->nt * sizeof(double));
        if (!rc) rc = dalloc((void**)&h->igamf, p->nt * sizeof(float));
        // The block fixed-point residual resolves the true residual of the FP64 iterate.  For stiff
        // problems (2^-24 dt max|spectrum| > 1) that residual's floor, the iterate's own rounding times
        // dt ||A||, lies above the usual tolerances, while the FP64 kernel's computed residual settles
        // lower (its rounding follows the iterate); there the FP64 kernel stays the default.
        h->use_fx = residual_fx_supported(h->geo) && stiffness_of(p) * 0x1p-24 <= 1.0;
    }
    if (!rc && p->precision == PINT_MIXED_FF) {
        rc = dalloc((void**)&h->Uff, z.dof * sizeof(float2));
        if (!rc) rc = dalloc((void**)&h->u0ff, z.nspace * sizeof(float2));
        if (!rc) rc = dalloc((void**)&h->gamf, p->nt * sizeof(float));
        if (!rc) rc = dalloc((void**)&h->ginvf, p->nt * sizeof(float));
    }
    if (!rc && f32_transforms(p) && time_gemm_supported(p->nt, (int)z.nspace)) {
        std::vector<uint16_t> wt;
        time_gemm_tables(p->nt, wt);
        rc = dalloc(&h->wgemm, wt.size() * sizeof(uint16_t));
        if (!rc && cudaMemcpyAsync(h->wgemm, wt.data(), wt.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, h->st) !=
                       cudaSuccess)
            rc = PINT_ECUDA;
        if (!rc) cudaStreamSynchronize(h->st);   // the host vector goes out of scope
    }
    if (!rc && !(h->hctl = ctl_slab_acquire())) rc = PINT_ENOMEM;
    if (!rc) rc = f32_transforms(p) ? build_tables<float>(h) : build_tables<double>(h);
    if (!rc && cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->st) != cudaSuccess) rc = PINT_ECUDA;
    if (rc) {
        pint_destroy(h);
        return rc;
    }
    h->npart = (int)z.partials;
    h->lev[0].nt = p->nt;
    h->lev[0].tabs = h->tabs_ptrs;
    h->lev[0].gam = h->gam;
    h->lev[0].ginv = h->ginv;
    h->lev[0].gamf = h->gamf;
    h->lev[0].ginvf = h->ginvf;
    h->lev[0].gdt = h->gdt;
    h->lev[0].igamf = h->igamf;
    h->nlev = 1;
    h->Uff_cur = h->Uff;
    {
        const int ny = p->dim == 2 ? p->ny : 1;
        h->lamx_h.resize(p->nx);
        h->lamy_h.resize(ny);
        for (int i = 0; i < p->nx; ++i) h->lamx_h[i] = lap_eig(i, p->nx, p->bc);
        for (int i = 0; i < ny; ++i) h->lamy_h[i] = p->dim == 2 ? lap_eig(i, ny, p->bc) : 0.0;
    }
    *out = h;
    return PINT_OK;
}

static int read_ctl(pint_handle* h) {
    PINT_CK(cudaMemcpyAsync(h->hctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st));
    PINT_CK(cudaStreamSynchronize(h->st));
    prof_flush(h);
    return PINT_OK;
}

int pint_profile_enable(pint_handle* h, int on) {
    if (!h || on < 0 || on > 2) return PINT_EINVAL;
    if (on && !h->ev[0]) {
        for (int i = 0; i < 2 * pint_handle::NEV; ++i)
            if (cudaEventCreate(&h->ev[i]) != cudaSuccess) return PINT_ECUDA;
    }
    PINT_CK(cudaStreamSynchronize(h->st));
    prof_flush(h);
    h->prof_on = on;
    return PINT_OK;
}

int pint_set_option(pint_handle* h, int option, long long value) {
    if (!h) return PINT_EINVAL;
    switch (option) {
        case PINT_OPT_GRAPHS:
            if (value != 0 && value != 1) return PINT_EINVAL;
            h->use_graphs = (int)value;
            return PINT_OK;
        case PINT_OPT_TIME_GEMM:
            if (value < -1 || value > 1) return PINT_EINVAL;
            if (value == 1 && !h->wgemm) return PINT_EINVAL;
            h->tgemm_mode = (int)value;
            h->tgemm_tuned = value >= 0 ? 1 : 0;
            h->gemm_fwd = h->gemm_inv = value == 1 ? 1 : 0;
            for (auto& sl : h->gslot)   // captured loops hold the old kernel choice
                if (sl.exec) { cudaGraphExecDestroy(sl.exec); sl.exec = nullptr; }
            return PINT_OK;
        case PINT_OPT_FX_RESIDUAL:
            if (value != 0 && value != 1) return PINT_EINVAL;
            if (value && !(h->p.precision == PINT_MIXED && residual_fx_supported(h->geo))) return PINT_EINVAL;
            h->use_fx = (int)value;
            for (auto& sl : h->gslot)   // captured loops hold the old kernel choice
                if (sl.exec) { cudaGraphExecDestroy(sl.exec); sl.exec = nullptr; }
            return PINT_OK;
        case PINT_OPT_FUSED_SPATIAL:
            if (value != 0 && value != 1) return PINT_EINVAL;
            h->fuse2d = (int)value;
            h->fuse2d_user = 1;
            for (auto& sl : h->gslot)   // captured loops hold the old kernel choice
                if (sl.exec) { cudaGraphExecDestroy(sl.exec); sl.exec = nullptr; }
            return PINT_OK;
        case PINT_OPT_KRYLOV: {
            if (value < 0 || value > kMaxKrylov) return PINT_EINVAL;
            if (value > 0 && h->coef.ch) return PINT_EINVAL;   // linear equations only
            const size_t dof = (size_t)h->p.nt * h->geo.nspace;
            for (double* q : {h->kv, h->kz, h->kzero, h->kpart, h->kcoef})
                if (q) cudaFreeAsync(q, h->st);
            h->kv = h->kz = h->kzero = h->kpart = h->kcoef = nullptr;
            h->krylov = 0;
            if (value == 0) return PINT_OK;
            auto al = [&](double** ptr, size_t count) {
                if (cudaMallocAsync((void**)ptr, count * sizeof(double), h->st) != cudaSuccess) {
                    cudaGetLastError();
                    return false;
                }
                return true;
            };
            if (!al(&h->kv, (value + 1) * dof) || !al(&h->kz, value * dof) || !al(&h->kzero, h->geo.nspace) ||
                !al(&h->kpart, (size_t)krylov_dot_blocks(dof) * (kMaxKrylov + 1)) || !al(&h->kcoef, kMaxKrylov + 1))
                return PINT_ENOMEM;
            if (cudaMemsetAsync(h->kzero, 0, h->geo.nspace * sizeof(double), h->st) != cudaSuccess) return PINT_ECUDA;
            h->krylov = (int)value;
            return PINT_OK;
        }
        case PINT_OPT_VARYING_JACOBIAN: {
            if (value < 0 || value > kMaxKrylov) return PINT_EINVAL;
            if (value > 0 && !h->coef.ch) return PINT_EINVAL;   // Cahn-Hilliard only
            for (auto& sl : h->gslot)   // captured loops hold the old Step 2
                if (sl.exec) { cudaGraphExecDestroy(sl.exec); sl.exec = nullptr; }
            for (void* q : {h->jbuf, h->jt, (void*)h->jpart, (void*)h->gmh, (void*)h->gmk})
                if (q) cudaFreeAsync(q, h->st);
            h->jbuf = h->jt = nullptr;
            h->jpart = nullptr;
            h->gmh = nullptr;
            h->gmk = nullptr;
            h->vary = 0;
            if (value == 0) return PINT_OK;
            const size_t tsz = f32_transforms(&h->p) ? 4 : 8;
            const int nk = h->p.nt / 2 + 1;
            const size_t n = (size_t)nk * h->geo.nspace;
            // partial sets of up to kMaxKrylov + 1 vectors, for every segment length (nbx nk <= 2*152*4 + nk)
            const size_t nparts = (size_t)cdot_blocks(h->geo.nspace, nk) * nk + 2 * 152 * 4 + nk;
            auto al = [&](void** ptr, size_t bytes) {
                if (cudaMallocAsync(ptr, bytes, h->st) != cudaSuccess) { cudaGetLastError(); return false; }
                return true;
            };
            if (!al(&h->jbuf, (size_t)(2 * value + 2) * n * 2 * tsz) || !al(&h->jt, h->geo.nspace * tsz) ||
                !al((void**)&h->jpart, nparts * (kMaxKrylov + 1) * 2 * sizeof(double)) ||
                !al((void**)&h->gmh, sizeof(GmHead)) || !al((void**)&h->gmk, (size_t)nk * sizeof(GmK)))
                return PINT_ENOMEM;
            h->vary = (int)value;
            return PINT_OK;
        }
        case PINT_OPT_LOG_INVARIANTS: {
            if (value != 0 && value != 1) return PINT_EINVAL;
            if (value && !h->inv_dev) {
                const size_t n = (size_t)h->p.n_windows * h->p.nt * 2;
                if (cudaMallocAsync((void**)&h->inv_dev, n * sizeof(double), h->st) != cudaSuccess) {
                    cudaGetLastError();
                    return PINT_ENOMEM;
                }
            }
            h->log_inv = (int)value;
            return PINT_OK;
        }
        case PINT_OPT_ADAPTIVE_WINDOWS: {
            if (value != 0 && value != 1) return PINT_EINVAL;
            if (value) {
                const int rc = f32_transforms(&h->p) ? build_levels<float>(h) : build_levels<double>(h);
                if (rc != PINT_OK) return rc;
            }
            h->adaptive = (int)value;
            return PINT_OK;
        }
        default: return PINT_EINVAL;
    }
}

int pint_profile_read(pint_handle* h, pint_profile* out, int reset) {
    if (!h || !out) return PINT_EINVAL;
    PINT_CK(cudaStreamSynchronize(h->st));
    prof_flush(h);
    for (int i = 0; i < PINT_NPHASE; ++i) {
        out->ms[i] = h->ms[i];
        out->launches[i] = h->launches[i];
        if (reset) { h->ms[i] = 0.0; h->launches[i] = 0; }
    }
    return PINT_OK;
}

// Adaptive window policy (PINT_OPT_ADAPTIVE_WINDOWS): the longest segment
// length L (a power of two, <= lmax) with alpha * G(L) <= 0.1, where
// G(L) = max_p R_p^L and R_p = 1/(1 + dt mu_p) over the spectrum mu_p of the
// spatial operator linearized about the segment's initial data (for
// Cahn-Hilliard mu(Lam) = eps^2 Lam^2 + (1 - jbar0) Lam with jbar0 = mean 3 u0^2;
// Eyre's splitting has its own factor, below).
// A mode with alpha R^L near 1 makes the iteration resonate (per-mode factor
// |alpha R^L / (1 - alpha R^L)|, Eq. 2.18), so growing modes force short segments.
static int choose_level(pint_handle* h, int lmax, double jbar0) {
    // per-step amplification of mode Lam of the scheme linearized about the data:
    //   backward Euler:  R = 1 / (1 + dt mu),  mu = c2 Lam^2 + c1 Lam (c1 = 1 - jbar0 for CH);
    //   Eyre splitting:  R = (1 - dt Lam) / (1 + dt (c2 Lam^2 - jbar0 Lam))
    const bool eyre = h->geo.expl != 0;
    const double dt = h->geo.dt, c2 = h->coef.c2, c1 = h->coef.ch ? h->coef.c1 - jbar0 : h->coef.c1;
    double lnR = 0.0;
    bool unstable = false;
    for (double lx : h->lamx_h)
        for (double ly : h->lamy_h) {
            const double L = lx + ly, den = 1.0 + dt * (c2 * L * L + c1 * L);
            if (den <= 0.0) { unstable = true; continue; }
            const double num = eyre ? 1.0 - dt * L : 1.0;
            lnR = fmax(lnR, log(fabs(num) / den));
        }
    int li = 0;
    while (li + 1 < h->nlev && h->lev[li].nt > lmax) ++li;
    if (unstable) return h->nlev - 1;
    if (lnR <= 0.0) return li;
    for (; li < h->nlev; ++li)
        if (log(h->p.alpha) + h->lev[li].nt * lnR <= log(0.1)) return li;
    return h->nlev - 1;
}

// Restarted flexible GMRES around P_alpha^{-1} (right preconditioning) for the
// linear equations: minimizes ||b - K U||_2 over U0 + span{P^{-1} v_j}, with
// K applied by the FP64 residual kernel (K z = -residual(z) at u0 = 0) and the
// preconditioner in the handle's precision.  Classical Gram-Schmidt applied
// twice; the preconditioned vectors are kept (flexible form), since complex64
// inner solves are not an exactly fixed linear map.  Fills hctl's status,
// iteration count (preconditioner applications), rho and history.
static int krylov_dots(pint_handle* h, const double* w, const double* V, int nv, size_t n, double* out) {
    const int nb = krylov_dot_blocks(n);
    launch_multi_dot(w, V, n, nv, n, h->kpart, h->st);
    std::vector<double> part((size_t)nb * nv);
    PINT_CK(cudaMemcpyAsync(part.data(), h->kpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    PINT_CK(cudaStreamSynchronize(h->st));
    for (int i = 0; i < nv; ++i) {
        double a = 0.0;
        for (int b = 0; b < nb; ++b) a += part[(size_t)b * nv + i];
        out[i] = a;
    }
    return PINT_OK;
}
static int krylov_axpy(pint_handle* h, double* w, const double* V, int nv, size_t n, const double* c) {
    PINT_CK(cudaMemcpyAsync(h->kcoef, c, nv * sizeof(double), cudaMemcpyHostToDevice, h->st));
    launch_multi_axpy(w, V, n, nv, h->kcoef, n, h->st);
    PINT_CK(cudaStreamSynchronize(h->st));   // c is host memory reused by the caller
    return PINT_OK;
}

static int gmres_window(pint_handle* h, double* U, const double* u0w) {
    const Geo& g = h->geo;
    const pint_problem& p = h->p;
    const size_t n = (size_t)g.nt * g.nspace;
    const int m = h->krylov;
    double* V = h->kv;
    double* Z = h->kz;
    int rc = read_ctl(h);
    if (rc != PINT_OK) return rc;
    const double bn = h->hctl->bnorm > 0.0 ? h->hctl->bnorm : 1.0;
    Ctl& c = *h->hctl;
    int iters = 0, nh = 0;
    auto record = [&](double rho) {
        if (nh < PINT_HIST_MAX) c.hist[nh] = rho;
        ++nh;
        c.rho = rho;
    };
    std::vector<double> H((size_t)(m + 1) * m, 0.0), gv(m + 1), cs(m), sn(m), y(m), hcol(m + 1), tmp(m + 1);
    for (;;) {
        // r0 = b - K U into v_0
        launch_residual<double>(g, U, u0w, nullptr, V, nullptr, h->partials, nullptr, h->st);
        double beta2;
        if ((rc = krylov_dots(h, V, V, 1, n, &beta2)) != PINT_OK) return rc;
        const double beta = sqrt(beta2);
        record(beta / bn);
        if (!(beta / bn == beta / bn)) { c.status = PINT_EDIVERGED; break; }
        if (beta / bn <= p.tol) { c.status = PINT_OK; break; }
        if (iters >= p.max_iter) { c.status = PINT_ENOCONV; break; }
        launch_scale_copy(V, V, 1.0 / beta, n, h->st);
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int j = 0;
        for (; j < m && iters < p.max_iter; ++j) {
            double* vj = V + (size_t)j * n;
            double* zj = Z + (size_t)j * n;
            double* w = V + (size_t)(j + 1) * n;
            cudaError_t e = f32_transforms(&h->p) ? Impl<float>::precond(h, 0.0, vj, zj) : Impl<double>::precond(h, 0.0, vj, zj);
            if (e != cudaSuccess) return PINT_ECUDA;
            ++iters;
            launch_residual<double>(g, zj, h->kzero, nullptr, w, nullptr, h->partials, nullptr, h->st);
            launch_scale_copy(w, w, -1.0, n, h->st);   // w = K z_j
            std::fill(hcol.begin(), hcol.end(), 0.0);
            for (int pass = 0; pass < 2; ++pass) {     // classical Gram-Schmidt, twice
                if ((rc = krylov_dots(h, w, V, j + 1, n, tmp.data())) != PINT_OK) return rc;
                for (int i = 0; i <= j; ++i) {
                    hcol[i] += tmp[i];
                    tmp[i] = -tmp[i];
                }
                if ((rc = krylov_axpy(h, w, V, j + 1, n, tmp.data())) != PINT_OK) return rc;
            }
            double hn2;
            if ((rc = krylov_dots(h, w, w, 1, n, &hn2)) != PINT_OK) return rc;
            hcol[j + 1] = sqrt(hn2);
            if (hcol[j + 1] > 0.0) launch_scale_copy(w, w, 1.0 / hcol[j + 1], n, h->st);
            // apply the previous Givens rotations to the new column, then a new one
            for (int i = 0; i < j; ++i) {
                const double a = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = a;
            }
            const double r = hypot(hcol[j], hcol[j + 1]);
            cs[j] = r > 0.0 ? hcol[j] / r : 1.0;
            sn[j] = r > 0.0 ? hcol[j + 1] / r : 0.0;
            hcol[j] = r;
            hcol[j + 1] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
            record(fabs(gv[j + 1]) / bn);
            if (fabs(gv[j + 1]) / bn <= p.tol) { ++j; break; }
        }
        // y = R^{-1} g (back substitution), U += Z y
        for (int i = j - 1; i >= 0; --i) {
            double a = gv[i];
            for (int k = i + 1; k < j; ++k) a -= H[(size_t)i * m + k] * y[k];
            y[i] = a / H[(size_t)i * m + i];
        }
        if (j > 0 && (rc = krylov_axpy(h, U, Z, j, n, y.data())) != PINT_OK) return rc;
        if (nh > 0) --nh;   // the true residual of the update is recorded at the top of the loop
    }
    c.iter = iters;   // preconditioner applications; hist holds one residual per application plus the first
    c.dnorm = 0.0;
    c.jbar = 0.0;
    return PINT_OK;
}

// Choose, by measurement on this handle's sizes, between the FFT kernels and the
// tensor-core DFT products for Step 1 and (PINT_MIXED) Step 3: each variant runs
// twice to warm up and five times timed with CUDA events on the handle's
// stream; the faster one is kept for the handle's life.
// Key of the autotuner table: the shape and the kernels' variant (precision as run).
static TuneKey tune_key(const pint_problem& p, const Geo& g) {
    TuneKey k{};
    k.equation = p.equation;
    k.dim = p.dim;
    k.nx = g.nx;
    k.ny = g.ny;
    k.nt = p.nt;
    k.precision = p.precision;
    k.bc = p.bc;
    k.half = p.theta < 1.0 ? 1 : 0;
    return k;
}

// The project autotuner, run before a handle's first solve: for each transform
// choice left to it (PINT_OPT_TIME_GEMM = -1: Step 1 and Step 3 as FFTs or as
// tensor-core DFT products; PINT_OPT_FUSED_SPATIAL not set by the caller: Step 2
// as one fused 2-D kernel or three passes) it times every candidate on this
// handle's buffers with CUDA events (two warm-up and five timed launches) and
// keeps the fastest.  The result goes into the process-wide table keyed by the
// problem's shape, so later handles of the same shape take it without measuring.
static int autotune(pint_handle* h) {
    h->tgemm_tuned = 1;
    const bool a_gemm = h->wgemm && time_gemm_supported(h->p.nt, h->geo.nspace);
    const bool a_fuse = h->geo.dim == 2 && slice2d_supported(h->geo, h->fft_x, h->fft_y, h->p.precision != PINT_FP64);
    const bool t_gemm = a_gemm && h->tgemm_mode == -1, t_fuse = a_fuse && !h->fuse2d_user;
    if (!t_gemm && !t_fuse) return PINT_OK;
    const TuneKey key = tune_key(h->p, h->geo);
    TuneVal v{};
    if (tune_lookup(key, &v)) {
        if (t_gemm) {
            h->gemm_fwd = v.gemm_fwd;
            h->gemm_inv = v.gemm_inv;
        }
        if (t_fuse) h->fuse2d = v.fused;
        h->tune_cached = 1;
        return PINT_OK;
    }
    const Geo& g = h->geo;
    const size_t dof = (size_t)g.nt * g.nspace;
    cudaEvent_t e0, e1;
    PINT_CK(cudaEventCreate(&e0));
    PINT_CK(cudaEventCreate(&e1));
    auto timeit = [&](auto fn) -> float {
        launch_set_running(h->ctl, 0.0, h->st);
        fn();
        fn();
        cudaEventRecord(e0, h->st);
        for (int i = 0; i < 5; ++i) fn();
        cudaEventRecord(e1, h->st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return cudaGetLastError() == cudaSuccess ? ms / 5.f : 1e30f;
    };
    float best = 0.f;
    v.gemm_fwd = h->gemm_fwd;
    v.gemm_inv = h->gemm_inv;
    v.fused = h->fuse2d;
    if (t_gemm) {
        double* tU = nullptr;
        if (cudaMallocAsync((void**)&tU, dof * sizeof(double), h->st) != cudaSuccess) {
            cudaGetLastError();
            tU = nullptr;   // keep the FFT
        }
        if (tU) {
            PINT_CK(cudaMemsetAsync(tU, 0, dof * sizeof(double), h->st));
            const Tabs<float>& tb = tabs_of<float>(h);
            float* s = reinterpret_cast<float*>(h->s);
            float2* S = reinterpret_cast<float2*>(h->S);
            const float ff = timeit([&] { launch_time_fwd<float>(g.nt, g.nspace, s, S, tb.twt, h->ctl, h->st); });
            const float gf = timeit([&] { launch_time_gemm(0, g.nt, g.nspace, s, S, h->wgemm, nullptr, h->ctl, nullptr, h->st); });
            v.gemm_fwd = gf < ff ? 1 : 0;
            best += gf < ff ? gf : ff;
            if (h->p.precision == PINT_MIXED) {
                const float fi = timeit([&] {
                    launch_time_inv<float>(g.nt, g.nspace, S, tb.twt, h->ginv, tU, 1, h->ctl, nullptr, h->st, h->s, nullptr);
                });
                const float gi = timeit([&] { launch_time_gemm(1, g.nt, g.nspace, S, tU, h->wgemm, h->ginv, h->ctl, nullptr, h->st); });
                v.gemm_inv = gi < fi ? 1 : 0;
                best += gi < fi ? gi : fi;
            }
            cudaFreeAsync(tU, h->st);
        }
        h->gemm_fwd = v.gemm_fwd;
        h->gemm_inv = v.gemm_inv;
    }
    if (t_fuse) {
        // Step 2 on a zeroed spectrum, fused and in three passes
        const bool f32 = f32_transforms(&h->p);
        PINT_CK(cudaMemsetAsync(h->S, 0, (size_t)(g.nt / 2 + 1) * g.nspace * 2 * (f32 ? 4 : 8), h->st));
        auto step2 = [&] {
            if (f32) Impl<float>::spatial(h, reinterpret_cast<float2*>(h->S), tabs_of<float>(h));
            else Impl<double>::spatial(h, reinterpret_cast<double2*>(h->S), tabs_of<double>(h));
        };
        h->fuse2d = 1;
        const float t1 = timeit(step2);
        h->fuse2d = 0;
        const float t3 = timeit(step2);
        v.fused = t1 <= t3 ? 1 : 0;
        h->fuse2d = v.fused;
        best += t1 <= t3 ? t1 : t3;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    PINT_CK(cudaStreamSynchronize(h->st));
    v.ms = best;
    // only a measurement of every choice this shape has is a table entry (none fixed by the caller)
    if (t_gemm == a_gemm && t_fuse == a_fuse) tune_store(key, v);
    return PINT_OK;
}

// The solve; with U_host, the device-to-host copy of the result is queued
// before the final synchronization, so it needs no round trip of its own.
static int solve_impl(pint_handle* h, const double* u0_dev, double* U_dev, pint_stats* st, double* U_host) {
    PINT_CK(cudaSetDevice(h->device));
    const pint_problem& p = h->p;
    const Geo& g = h->geo;
    const bool kry = h->krylov > 0;   // outer GMRES: FP64 iterate in U_dev (a float-float request acts as mixed)
    const bool ffm = p.precision == PINT_MIXED_FF && !kry;
    const int ntmax = h->lev[0].nt;
    const size_t ns = (size_t)g.nspace, dof = (size_t)ntmax * ns;
    const bool adapt = h->adaptive && h->nlev > 1 && p.theta == 1.0;   // the policy's growth factor is BE's
    pint_stats S;
    memset(&S, 0, sizeof(S));
    S.nt_min = ntmax;
    int rc = PINT_OK;
    bool converted = false;   // float-float result already converted to U_dev
    activate_level(h, 0);
    if (!h->tgemm_tuned && (rc = autotune(h)) != PINT_OK) return rc;
    // Cahn-Hilliard never starts from the zero iterate: its scalar Jacobian
    // 3 mean(u^2) would be 0 in the first preconditioner, far from the state's,
    // and the iteration can diverge; such windows start from u0 instead.
    const int init = (p.init_guess == 2 && h->coef.ch) ? 0 : p.init_guess;
    if (ffm && init == 1) launch_f64_to_ff(U_dev, h->Uff, dof, h->st);
    const long long total = (long long)ntmax * p.n_windows;
    long long done = 0;
    h->inv_count = 0;
    for (int seg = 0; done < total; ++seg) {
        const int base = (int)(done % ntmax);   // offset of this segment inside its window
        const double* u0w = seg == 0 ? u0_dev : h->u0buf;
        prof_begin(h, PH_SETUP);
        int nl = 0;
        if (ffm && seg == 0) { launch_f64_to_ff(u0_dev, h->u0ff, g.nspace, h->st); nl++; }
        if (adapt) nl += 2;
        int li = 0;
        if (adapt) {
            // segments never cross a window boundary: at offset base the length
            // is at most the largest power of two dividing base
            const int lmax = base == 0 ? ntmax : (base & -base);
            activate_level(h, 0);
            launch_begin_window(g, u0w, p.max_iter, p.tol, h->partials, h->ctl, h->st, p.tol_update, h->b1);
            if ((rc = read_ctl(h)) != PINT_OK) return rc;
            const double rms = h->hctl->bnorm * g.dt;          // ||u0||_2
            li = choose_level(h, lmax, 3.0 * rms * rms / (double)ns);
        }
        prof_end(h, PH_SETUP, nl);
        double* Useg = U_dev + (size_t)base * ns;
        int L = 0;
        // Solve the segment; under the adaptive policy a segment that diverges
        // or stalls is solved again from the same initial data with half the length.
        for (bool first_try = true;; first_try = false) {
            activate_level(h, li);
            L = g.nt;
            h->Uff_cur = ffm ? h->Uff + (size_t)base * ns : h->Uff;
            const size_t sdof = (size_t)L * ns;
            prof_begin(h, PH_SETUP);
            nl = 1;
            if (init == 2) {
                PINT_CK(ffm ? cudaMemsetAsync(h->Uff_cur, 0, sdof * sizeof(float2), h->st)
                            : cudaMemsetAsync(Useg, 0, sdof * sizeof(double), h->st));
            } else if (seg > 0 || init == 0 || !first_try) {
                if (ffm) launch_broadcast_ff(h->Uff_cur, h->u0ff, g.nspace, L, h->st);
                else launch_broadcast(Useg, u0w, g.nspace, L, h->st);
                nl++;
            }
            launch_begin_window(g, u0w, p.max_iter, p.tol, h->partials, h->ctl, h->st, p.tol_update, h->b1);
            prof_end(h, PH_SETUP, nl + 1);
            cudaGraphExec_t gx = (h->use_graphs && !h->prof_on && !adapt && !kry) ? get_graph(h, Useg, u0w) : nullptr;
            if (kry) {
                if ((rc = gmres_window(h, Useg, u0w)) != PINT_OK) return rc;
            } else if (gx) {
                // one graph launch runs the iteration loop of this window to its stop
                if (init == 2 && zero_start(h, Useg, u0w) != cudaSuccess) return PINT_ECUDA;
                PINT_CK(cudaGraphLaunch(gx, h->st));
                if (ffm && done + L >= total) {
                    // the last window: queue the result's conversion (and copy) ahead of the
                    // status read, so that one synchronization covers all of it
                    launch_ff_to_f64(h->Uff, U_dev, dof, h->st);
                    h->launches[PH_SETUP] += 1;
                    converted = true;
                    if (U_host) PINT_CK(cudaMemcpyAsync(U_host, U_dev, dof * sizeof(double), cudaMemcpyDeviceToHost, h->st));
                }
                if ((rc = read_ctl(h)) != PINT_OK) return rc;
                if (h->hctl->status == ST_RUNNING) return PINT_ECUDA;  // the loop ends only on a final status
                const long long runs = h->hctl->iter + 1 - (init == 2 ? 1 : 0);
                h->launches[PH_RES] += runs;
                h->launches[PH_CHECK] += runs;
                h->launches[PH_TFWD] += runs * (use_gemm_fwd(h) ? 1 : time_fwd_launches(g.nt));
                for (int stg = 0; stg < spatial_launches(h); ++stg) h->launches[PH_SP0 + stg] += runs;
                h->launches[PH_TINV] += runs * (use_gemm_inv(h) ? 1 : time_inv_launches(g.nt));
            } else {
                int enqueued = 0;
                for (;;) {
                    int chunk = enqueued == 0 ? 3 : 2;
                    for (int c = 0; c < chunk; ++c) {
                        cudaError_t e = enqueued == 0 && c == 0 && init == 2 ? zero_start(h, Useg, u0w)
                                        : ffm ? iteration_ff(h) : iteration(h, Useg, u0w);
                        if (e != cudaSuccess) return PINT_ECUDA;
                    }
                    enqueued += chunk;
                    if ((rc = read_ctl(h)) != PINT_OK) return rc;
                    if (h->hctl->status != ST_RUNNING) break;
                    if (enqueued > p.max_iter + 8) return PINT_ECUDA;  // the device loop must have stopped by now
                }
            }
            const int stt = h->hctl->status;
            S.iters += h->hctl->iter;
            if (adapt && stt != PINT_OK && li + 1 < h->nlev) {
                ++li;
                ++S.retries;
                continue;
            }
            break;
        }
        const Ctl& c = *h->hctl;
        const int k = c.iter;
        S.status = c.status;
        S.iters_last = k;
        S.segments = seg + 1;
        if (L < S.nt_min) S.nt_min = L;
        S.rel_residual = c.rho;
        S.update_norm = p.tol_update > 0.0 ? c.dnorm : 0.0;
        S.precision = p.precision;
        S.time_gemm = (use_gemm_fwd(h) ? 1 : 0) | (use_gemm_inv(h) ? 2 : 0);
        S.fused_spatial = fused_spatial(h) ? 1 : 0;
        S.tune_cached = h->tune_cached;
        S.jbar = h->coef.ch ? c.jbar : 0.0;
        for (int i = 0; i <= k && i < PINT_HIST_MAX; ++i) S.hist[i] = c.hist[i];
        S.contraction = k >= 2 ? pow(c.hist[k] / c.hist[1], 1.0 / (k - 1)) : (k == 1 ? c.hist[1] / c.hist[0] : 0.0);
        if (c.status != PINT_OK) {
            rc = c.status;
            break;
        }
        if (h->log_inv) {
            // mass and discrete energy of the segment's L levels (time levels done+1 .. done+L)
            const double hh = grid_h(p.nx, p.bc);
            if (ffm) launch_invariants<float2>(h->Uff_cur, L, g, p.eps, hh, h->inv_dev + 2 * done, h->st);
            else launch_invariants<double>(Useg, L, g, p.eps, hh, h->inv_dev + 2 * done, h->st);
            h->launches[PH_SETUP] += 1;
            h->inv_count = done + L;
        }
        done += L;
        S.windows = (int)(done / ntmax);
        if (done < total) {
            if (ffm) {
                PINT_CK(cudaMemcpyAsync(h->u0ff, h->Uff_cur + (size_t)(L - 1) * ns, ns * sizeof(float2),
                                        cudaMemcpyDeviceToDevice, h->st));
                launch_ff_to_f64(h->u0ff, h->u0buf, g.nspace, h->st);
            } else {
                PINT_CK(cudaMemcpyAsync(h->u0buf, Useg + (size_t)(L - 1) * ns, ns * sizeof(double),
                                        cudaMemcpyDeviceToDevice, h->st));
            }
        }
    }
    activate_level(h, 0);
    h->Uff_cur = h->Uff;
    if (!converted) {
        if (ffm) {
            launch_ff_to_f64(h->Uff, U_dev, dof, h->st);
            h->launches[PH_SETUP] += 1;
        }
        if (U_host) PINT_CK(cudaMemcpyAsync(U_host, U_dev, dof * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    }
    PINT_CK(cudaStreamSynchronize(h->st));
    if (st) *st = S;
    return rc;
}

int pint_solve(pint_handle* h, const double* u0_dev, double* U_dev, pint_stats* st) {
    if (!h || !u0_dev || !U_dev) return PINT_EINVAL;
    return solve_impl(h, u0_dev, U_dev, st, nullptr);
}

int pint_solve_batch(pint_handle* const* hs, int n, const double* const* u0s, double* const* Us, pint_stats* st,
                     int* rcs) {
    if (n < 0 || (n > 0 && (!hs || !u0s || !Us))) return PINT_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!hs[i] || !u0s[i] || !Us[i]) return PINT_EINVAL;
    std::vector<int> rc(n, PINT_OK);
    std::atomic<int> next{0};
    auto work = [&]() {
        for (int i; (i = next.fetch_add(1)) < n;) rc[i] = pint_solve(hs[i], u0s[i], Us[i], st ? &st[i] : nullptr);
    };
    const int workers = n < 64 ? n : 64;
    std::vector<std::thread> th;
    for (int w = 1; w < workers; ++w) th.emplace_back(work);
    if (n > 0) work();
    for (auto& t : th) t.join();
    int first = PINT_OK;
    for (int i = 0; i < n; ++i) {
        if (rcs) rcs[i] = rc[i];
        if (first == PINT_OK && rc[i] != PINT_OK) first = rc[i];
    }
    return first;
}

int pint_solve_host(pint_handle* h, const double* u0_host, double* U_host, pint_stats* st) {
    if (!h || !u0_host || !U_host) return PINT_EINVAL;
    const size_t ns = (size_t)h->geo.nspace, dof = ns * h->geo.nt;
    if (!h->hU) {
        if (cudaMallocAsync((void**)&h->hU, dof * sizeof(double), h->st) != cudaSuccess) { cudaGetLastError(); return PINT_ENOMEM; }
        if (cudaMallocAsync((void**)&h->hu0, ns * sizeof(double), h->st) != cudaSuccess) { cudaGetLastError(); return PINT_ENOMEM; }
    }
    PINT_CK(cudaMemcpyAsync(h->hu0, u0_host, ns * sizeof(double), cudaMemcpyHostToDevice, h->st));
    if (h->p.init_guess == 1)
        PINT_CK(cudaMemcpyAsync(h->hU, U_host, dof * sizeof(double), cudaMemcpyHostToDevice, h->st));
    return solve_impl(h, h->hu0, h->hU, st, U_host);
}

int pint_residual(pint_handle* h, const double* u0_dev, const double* U_dev, double* r_dev, double* rel_res) {
    if (!h || !u0_dev || !U_dev) return PINT_EINVAL;
    const Geo& g = h->geo;
    launch_begin_window(g, u0_dev, h->p.max_iter, h->p.tol, h->partials, h->ctl, h->st);
    int gx, gy, gz, chunk, np;
    if (h->use_fx) {
        PINT_CK(launch_residual_fx(h->gfx, g, U_dev, u0_dev, nullptr, nullptr, nullptr, r_dev, h->partials, nullptr,
                                   h->st, 1));
        np = residual_fx_grid(g, gx, gy, gz, chunk);
    } else {
        launch_residual<double>(g, U_dev, u0_dev, h->gam, r_dev, nullptr, h->partials, nullptr, h->st);
        np = residual_grid(g, gx, gy, gz, chunk);
    }
    launch_residual_norm(h->partials, np, h->ctl, h->st);
    PINT_CK(cudaGetLastError());
    int rc = read_ctl(h);
    if (rc != PINT_OK) return rc;
    if (rel_res) *rel_res = h->hctl->rho;
    return PINT_OK;
}

int pint_invariants(pint_handle* h, double* mass_host, double* energy_host, long long cap) {
    if (!h || cap < 0 || (cap > 0 && (!mass_host || !energy_host))) return PINT_EINVAL;
    if (!h->log_inv || !h->inv_dev) return PINT_EINVAL;
    const long long n = h->inv_count < cap ? h->inv_count : cap;
    if (n > 0) {
        std::vector<double> buf((size_t)n * 2);
        PINT_CK(cudaMemcpyAsync(buf.data(), h->inv_dev, buf.size() * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        PINT_CK(cudaStreamSynchronize(h->st));
        for (long long i = 0; i < n; ++i) {
            mass_host[i] = buf[2 * i];
            energy_host[i] = buf[2 * i + 1];
        }
    }
    return (int)(h->inv_count > 0x7fffffff ? 0x7fffffff : h->inv_count);
}

int pint_precond_apply(pint_handle* h, double jbar, const double* r_dev, double* delta_dev) {
    if (!h || !r_dev || !delta_dev || r_dev == delta_dev) return PINT_EINVAL;
    cudaError_t e = f32_transforms(&h->p) ? Impl<float>::precond(h, jbar, r_dev, delta_dev)
                                                  : Impl<double>::precond(h, jbar, r_dev, delta_dev);
    if (e != cudaSuccess) return PINT_ECUDA;
    PINT_CK(cudaStreamSynchronize(h->st));
    return PINT_OK;
}

int pint_tune_lookup(const pint_problem* p, pint_tune_entry* out) {
    if (!p || validate(p) != PINT_OK) return PINT_EINVAL;
    pint_problem q = *p;
    q.precision = effective_precision(p);
    Geo g;
    geometry_of(&q, g);
    TuneVal v{};
    if (!tune_lookup(tune_key(q, g), &v)) return 0;
    if (out) {
        out->time_fwd_gemm = v.gemm_fwd;
        out->time_inv_gemm = v.gemm_inv;
        out->fused_spatial = v.fused;
        out->ms = v.ms;
    }
    return 1;
}

int pint_tune_load(const char* path) {
    if (!path) return PINT_EINVAL;
    const int n = tune_load(path);
    return n < 0 ? PINT_EINVAL : n;
}

int pint_tune_save(const char* path) {
    if (!path) return PINT_EINVAL;
    const int n = tune_save(path);
    return n < 0 ? PINT_EINVAL : n;
}

void pint_tune_clear(void) { tune_clear(); }

}  // extern "C"
