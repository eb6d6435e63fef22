// pint_static.cu - pint_residual_static: the all-at-once residual and its
// relative norm for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc at the moment they need a
// residual: code that runs while a framework's caching allocator has already
// reserved the whole device, code on a latency path that must never block in
// the allocator, or a process whose device memory is fixed once at start-up.
// For them this entry point needs no handle and allocates nothing: its
// reduction scratch is the file-scope array below, which lives in every GPU
// that loads the library until the process exits.
#include <mutex>

#include "../../include/pint.h"
#include "pint_common.cuh"
#include "pint_kernels.h"

namespace pint {

// Scratch: a control block (||b||, sums) followed by the per-CTA partial sums
// of the residual kernel.  Size: PINT_STATIC_SCRATCH_BYTES.
static __device__ __align__(256) unsigned char g_static_scratch[PINT_STATIC_SCRATCH_BYTES];

static constexpr size_t kCtlBytes = (sizeof(Ctl) + 255) / 256 * 256;
static constexpr size_t kMaxPairs = (PINT_STATIC_SCRATCH_BYTES - kCtlBytes) / (2 * sizeof(double));
// The largest residual grid pint_create accepts: a 2-D grid of 4096 x 1024 points (the largest
// FFT axes) in 32 x 8 tiles with all time levels in one CTA, 128 * 128 CTAs; 1-D grids need at
// most about 4 x 152.  Every accepted problem therefore fits the scratch.
static constexpr size_t kLargestResidualGrid = (4096 / 32) * (1024 / 8);
static_assert(kMaxPairs >= kLargestResidualGrid, "static scratch too small for the largest residual grid");

// ||r|| / ||b|| from the residual's partial sums and ctl->bnorm, written to out.
__global__ void k_static_finish(const double* __restrict__ partials, int np, const Ctl* __restrict__ ctl,
                                double* __restrict__ out) {
    __shared__ double ra[8];
    double a = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) a += partials[2 * i];
    a = warp_sum(a);
    if (threadIdx.x % 32 == 0) ra[threadIdx.x / 32] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0;
        for (int w = 0; w < 8; ++w) A += ra[w];
        const double bn = ctl->bnorm;
        *out = bn > 0.0 ? sqrt(A) / bn : sqrt(A);
    }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and reused by every later call.
static void* scratch_address(int& err) {
    static std::mutex mu;
    static void* addr[128] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        err = PINT_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            err = PINT_ECUDA;
            return nullptr;
        }
        addr[dev] = p;
    }
    err = PINT_OK;
    return addr[dev];
}

int validate_problem(const pint_problem* p);
void geometry_of(const pint_problem* p, Geo& g);

}  // namespace pint

using namespace pint;

extern "C" int pint_residual_static(const pint_problem* p, void* cuda_stream, const double* u0_dev,
                                    const double* U_dev, double* r_dev, double* rel_res_dev) {
    if (!u0_dev || !U_dev || !rel_res_dev) return PINT_EINVAL;
    int rc = validate_problem(p);
    if (rc != PINT_OK) return rc;
    Geo g;
    geometry_of(p, g);
    int gx, gy, gz, chunk;
    const int np = residual_grid(g, gx, gy, gz, chunk);
    const int nb = norm2_blocks(g.nspace);
    if ((size_t)np > kMaxPairs || (size_t)nb > kMaxPairs) return PINT_EINVAL;  // grid too large for the scratch
    void* base = scratch_address(rc);
    if (!base) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Ctl* ctl = reinterpret_cast<Ctl*>(base);
    double* partials = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(base) + kCtlBytes);
    // ||b|| = ||u0|| / dt: writes nb partial pairs, then ctl->bnorm (and resets ctl's other fields)
    launch_begin_window(g, u0_dev, p->max_iter, p->tol, partials, ctl, st);
    // residual: overwrites np partial pairs (every pair read below is written first)
    launch_residual<double>(g, U_dev, u0_dev, nullptr, r_dev, nullptr, partials, nullptr, st);
    k_static_finish<<<1, 256, 0, st>>>(partials, np, ctl, rel_res_dev);
    return cudaGetLastError() == cudaSuccess ? PINT_OK : PINT_ECUDA;
}
