// acac_residual_noalloc: the nonlinear residual F(X1) without a handle and without
// any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a residual:
// code that runs inside a host framework that owns every device allocation (a
// memory pool or arena that forbids stray cudaMalloc calls), latency-critical loops
// that must not block on the allocator, or plugins that are handed only the input
// and output buffers.  For them this entry point keeps its working memory (the
// per-cell variational derivative and mobility, the partial sums of ||F||^2 and
// the admissibility flags) in arrays with static storage in this file.  The
// arrays exist once per GPU that loads the library and stay allocated until the
// process exits; the grid is limited to NOALLOC_MAX_CELLS cells.
//
// The first call on a device looks up the arrays' device addresses with
// cudaGetSymbolAddress (host code cannot use the array names as device pointers) and
// caches them per device for the life of the process; make that first call before any
// stream capture.  Every call reads ||F||^2 and a flag back to the host and synchronises
// its stream.  All calls share the arrays, so calls whose work overlaps on the GPU
// (other streams, other host threads) race.  A cudaDeviceReset invalidates the cached
// addresses; the library does not support use across a device reset.
#include <mutex>
#include <string.h>

#include "acac_internal.cuh"

namespace acac {
namespace {

constexpr int NOALLOC_MAX_CELLS = 512 * 512;
constexpr size_t NOALLOC_G = 3 * (size_t)NOALLOC_MAX_CELLS;          // [G_u | G_v | c]
constexpr size_t NOALLOC_DOUBLES = NOALLOC_G + RED_BLOCKS + 32;      // + partials + result

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];
static __device__ __align__(256) int g_noalloc_flags[8];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double* g_scratch_ptr[MAX_DEVICES];
int* g_flags_ptr[MAX_DEVICES];

// Device addresses of the static arrays on the current device (looked up once).
int device_scratch(double** scratch, int** flags) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ACAC_E_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return ACAC_E_ARG;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* s = nullptr;
        void* f = nullptr;
        if (cudaGetSymbolAddress(&s, g_noalloc_scratch) != cudaSuccess) return ACAC_E_CUDA;
        if (cudaGetSymbolAddress(&f, g_noalloc_flags) != cudaSuccess) return ACAC_E_CUDA;
        g_scratch_ptr[dev] = static_cast<double*>(s);
        g_flags_ptr[dev] = static_cast<int*>(f);
    }
    *scratch = g_scratch_ptr[dev];
    *flags = g_flags_ptr[dev];
    return ACAC_OK;
}

}  // namespace
}  // namespace acac

extern "C" int acac_residual_noalloc(const acac_params* p, const double* X1, const double* X0, double dt,
                                     double* F, double* fnorm, void* cuda_stream) {
    using namespace acac;
    if (!p || !X1 || !X0 || !F || !(dt > 0)) return ACAC_E_ARG;
    int st = validate_params(p);
    if (st != ACAC_OK) return st;
    const long long ncell = (long long)p->n[0] * p->n[1] * (p->dim == 3 ? p->n[2] : 1);
    if (ncell > NOALLOC_MAX_CELLS) return ACAC_E_ARG;
    double* scratch = nullptr;
    int* flags = nullptr;
    st = device_scratch(&scratch, &flags);
    if (st != ACAC_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    const Geom g = make_geom(p);
    const Coef k{p->alpha, p->beta, p->theta, p->gamma, p->rho, p->taylor_S};

    // the flags accumulate with atomicOr: clear them for this call (flags[4] is the
    // reduction counter: zero between calls, re-armed by the kernel; clearing it too
    // recovers from an earlier call that failed mid-way)
    if (cudaMemsetAsync(flags, 0, 8 * sizeof(int), s) != cudaSuccess) return ACAC_E_CUDA;
    ResidualArgs a;
    a.X = X1; a.S = nullptr; a.lam = 0.0; a.shift = 0.0; a.X0 = X0; a.dt = dt;
    double* result = scratch + NOALLOC_G + RED_BLOCKS;
    a.Xt = nullptr; a.G = scratch; a.F = F; a.flags = flags;
    a.red = Red{scratch + NOALLOC_G, result, reinterpret_cast<unsigned*>(flags + 4)};
    if (launch_residual_g(g, k, a, s) != cudaSuccess) return ACAC_E_CUDA;
    if (launch_residual_f(g, k, a, s) != cudaSuccess) return ACAC_E_CUDA;
    double f2 = 0.0;
    int fl = 0;
    if (cudaMemcpyAsync(&f2, result, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ACAC_E_CUDA;
    if (cudaMemcpyAsync(&fl, flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ACAC_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ACAC_E_CUDA;
    if (fnorm) *fnorm = sqrt(f2);
    return (fl & 1) ? ACAC_E_DOMAIN : ACAC_OK;
}
