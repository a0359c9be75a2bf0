// Internal definitions of the acac CUDA library (sm_103a).
//
// Data layout in HBM (one GPU, one problem):
//   * a field is N = nx*ny doubles, x fastest;
//   * a state / residual / Krylov vector is [u field | v field] (2N values);
//   * the linearisation cache holds 7 fields per cell (c, dc/du1, dc/dv1, G_u, G_v,
//     dG_u/du1 pointwise part, dG_u/dv1 pointwise part) in Krylov precision;
//   * the assembled Jacobian is stencil-diagonal: 13 slots x 4 entries x N;
//   * ILU factors: per subdomain, level-major (wavefront level i + 2j), and inside a
//     level coefficient-major ([52][cells of the level]) so that the threads of one
//     level read consecutive addresses.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <vector>

#include "../../include/acac.h"

namespace acac {

constexpr int NSLOT = 13;          // radius-2 stencil (|o|_1 <= 2) in 2D
constexpr int NCOEF = 56;          // stored per cell: forward record + backward record
constexpr int CREC = 28;           // record: 6 lower 2x2 blocks (+4 pad) | inverse pivot + 6 upper blocks
constexpr int MAX_S = 30;          // Lemma 2.2 series terms accepted
constexpr int MAX_RESTART = 64;
constexpr int RED_BLOCKS = 1216;   // 152 SMs x 8: partial-sum blocks of the reductions
constexpr int RED_THREADS = 256;
constexpr int RAS_MAXBUF = 16;    // coefficient stages of the Schwarz apply ring

// Stencil slot order (dx, dy); mirrored in include/acac.h for acac_jacobian.
__host__ __device__ constexpr int slot_dx(int s) {
    return s == 1 ? -1 : s == 2 ? 1 : s == 5 ? -2 : s == 6 ? 2 : (s == 9 || s == 11) ? -1
         : (s == 10 || s == 12) ? 1 : 0;
}
__host__ __device__ constexpr int slot_dy(int s) {
    return s == 3 ? -1 : s == 4 ? 1 : s == 7 ? -2 : s == 8 ? 2 : (s == 9 || s == 10) ? -1
         : (s == 11 || s == 12) ? 1 : 0;
}
// Slot of offset (dx, dy), -1 if outside the stencil.
__host__ __device__ constexpr int slot_of(int dx, int dy) {
    return (dx == 0 && dy == 0) ? 0 : (dx == -1 && dy == 0) ? 1 : (dx == 1 && dy == 0) ? 2
         : (dx == 0 && dy == -1) ? 3 : (dx == 0 && dy == 1) ? 4 : (dx == -2 && dy == 0) ? 5
         : (dx == 2 && dy == 0) ? 6 : (dx == 0 && dy == -2) ? 7 : (dx == 0 && dy == 2) ? 8
         : (dx == -1 && dy == -1) ? 9 : (dx == 1 && dy == -1) ? 10 : (dx == -1 && dy == 1) ? 11
         : (dx == 1 && dy == 1) ? 12 : -1;
}
// Lower neighbours in increasing natural (x fastest) order, and upper neighbours.
__host__ __device__ constexpr int lower_dx(int k) { return k == 0 ? 0 : k == 1 ? -1 : k == 2 ? 0 : k == 3 ? 1 : k == 4 ? -2 : -1; }
__host__ __device__ constexpr int lower_dy(int k) { return k == 0 ? -2 : k <= 3 ? -1 : 0; }
__host__ __device__ constexpr int upper_dx(int k) { return k == 0 ? 1 : k == 1 ? 2 : k == 2 ? -1 : k == 3 ? 0 : k == 4 ? 1 : 0; }
__host__ __device__ constexpr int upper_dy(int k) { return k <= 1 ? 0 : k <= 4 ? 1 : 2; }

// Face directions of a cell: -x, +x, -y, +y.
__host__ __device__ constexpr int face_dx(int f) { return f == 0 ? -1 : f == 1 ? 1 : 0; }
__host__ __device__ constexpr int face_dy(int f) { return f == 2 ? -1 : f == 3 ? 1 : 0; }

struct Geom {
    int nx, ny, N;
    int bc;              // ACAC_BC_*
    double hx, hy;
    double ihx2, ihy2;   // 1/hx^2, 1/hy^2
    double vol;          // hx*hy
    float ihx2f, ihy2f;  // the same in float, for the FP32 Jacobian kernels
};

struct Coef {
    double alpha, beta, theta, gamma, rho;
    int S;
};

// Neighbour index of (x+dx, y+dy): wrapped (periodic) or clamped (Neumann; the
// clamped value is the ghost of Sec. 2, phi_0 = phi_1).
__device__ __forceinline__ int nb_index(const Geom& g, int x, int y, int dx, int dy) {
    int xx = x + dx, yy = y + dy;
    if (g.bc == ACAC_BC_PERIODIC) {
        xx = xx < 0 ? xx + g.nx : (xx >= g.nx ? xx - g.nx : xx);
        yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
    } else {
        xx = xx < 0 ? 0 : (xx >= g.nx ? g.nx - 1 : xx);
        yy = yy < 0 ? 0 : (yy >= g.ny ? g.ny - 1 : yy);
    }
    return yy * g.nx + xx;
}
// 1 if face f of cell (x, y) carries flux (always when periodic; interior faces
// only when Neumann: zero flux through the wall).
__device__ __forceinline__ double face_open(const Geom& g, int x, int y, int f) {
    if (g.bc == ACAC_BC_PERIODIC) return 1.0;
    int xx = x + face_dx(f), yy = y + face_dy(f);
    return (xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny) ? 1.0 : 0.0;
}
// 1/h^2 of face f of cell (x, y) if it carries flux, else 0, in precision T.
template <typename T>
__device__ __forceinline__ T face_w(const Geom& g, int x, int y, int f);
template <>
__device__ __forceinline__ double face_w<double>(const Geom& g, int x, int y, int f) {
    int xx = x + face_dx(f), yy = y + face_dy(f);
    const bool open = g.bc == ACAC_BC_PERIODIC || (xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny);
    return open ? (f < 2 ? g.ihx2 : g.ihy2) : 0.0;
}
template <>
__device__ __forceinline__ float face_w<float>(const Geom& g, int x, int y, int f) {
    int xx = x + face_dx(f), yy = y + face_dy(f);
    const bool open = g.bc == ACAC_BC_PERIODIC || (xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny);
    return open ? (f < 2 ? g.ihx2f : g.ihy2f) : 0.0f;
}
__device__ __forceinline__ bool in_domain(const Geom& g, int x, int y) {
    return g.bc == ACAC_BC_PERIODIC || (x >= 0 && x < g.nx && y >= 0 && y < g.ny);
}

// Linearisation cache (Krylov precision T).  For cell k:
//   c, cu = dc/du1, cv = dc/dv1, Gu, Gv, du = dG_u/du1 pointwise part
//   (-alpha/2 + theta dphi/dp1 + theta dpsi/dq1), xc = theta (dphi/dp1 - dpsi/dq1).
//   dG_v/dv1 pointwise part = du + (alpha - beta)/2.
template <typename T>
struct Cache {
    T* c; T* cu; T* cv; T* Gu; T* Gv; T* du; T* xc;
};

// One subdomain of the Schwarz decomposition (Sec. 3.1).
struct SubInfo {
    int ox, oy;          // global coordinates of the box corner (may be < 0 when periodic)
    int W, H;            // box size
    int own_x0, own_x1;  // owned (non-overlapping) range, box-local
    int own_y0, own_y1;
    int nlev;            // wavefront levels = (W-1) + 2(H-1) + 1
    int lev_base;        // first entry of this subdomain in the level-offset table
    long long coef_base; // first coefficient of this subdomain
    long long vec_base;  // first padded-vector element in the global scratch
};

// Row pitch (in cells) of a padded box vector: W + 4, made odd so that the cells of
// one wavefront level (row stride pitch - 2) fall into distinct shared-memory banks.
__host__ __device__ constexpr int ras_pitch(int W) { return (W + 4) | 1; }

// Shared-memory plan of the Schwarz apply kernel (bytes / elements).
struct RasLaunch {
    int nbuf;            // coefficient stages in flight
    int threads;         // consumer warps (2 threads per cell of the widest level) + 1 producer warp
    int stage_elems;     // elements per stage (>= 28 x the largest level)
    int stage_off;       // byte offset of the stages (after mbarriers and level table)
    int vec_off;         // byte offset of the box vector when it is in shared memory
    size_t smem_bytes;   // dynamic shared memory per CTA
};

// Checks of acac_create (sizes, coefficients, partition, enumerations).
int validate_params(const acac_params* p);

// ---------------------------------------------------------------- kernels (launchers)
// residual.cu
cudaError_t set_taylor_constants(int S);
struct ResidualArgs {
    const double* X;     // state at which F is evaluated (the trial state in a line search)
    const double* S;     // direction (trial_kernel only)
    double lam, shift;   // trial u = X_u + lam (S_u + shift), v = X_v + lam S_v
    const double* X0;
    double dt;
    double* Xt;          // trial state written by trial_kernel
    double* G;           // [Gu | Gv | c], 3N
    double* F;           // residual
    double* partial;     // RED_BLOCKS partial sums of F^2
    int* flags;          // bit 0: midpoint inadmissible, bit 1: trial state inadmissible
};
cudaError_t launch_residual_g(const Geom& g, const Coef& k, const ResidualArgs& a, cudaStream_t s);
cudaError_t launch_residual_f(const Geom& g, const Coef& k, const ResidualArgs& a, cudaStream_t s);
cudaError_t launch_trial(const Geom& g, const ResidualArgs& a, cudaStream_t s);
cudaError_t launch_table_log(const double* x, double* y, long long n, cudaStream_t s);
cudaError_t launch_energy(const Geom& g, const Coef& k, const double* X, double* partial,
                          int* flags, cudaStream_t s);
template <typename T>
cudaError_t launch_linearize(const Geom& g, const Coef& k, const double* X, const double* X0,
                             const double* G, Cache<T> cache, cudaStream_t s);

// jacobian.cu
template <typename T>
cudaError_t launch_assemble(const Geom& g, const Coef& k, double dt, Cache<T> cache, T* J,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_spmv(const Geom& g, const T* J, const T* w, T* y, cudaStream_t s);
template <typename T>
cudaError_t launch_jvp_g(const Geom& g, const Coef& k, Cache<T> cache, const T* w, T* tmp,
                         cudaStream_t s);
template <typename T>
cudaError_t launch_jvp_f(const Geom& g, const Coef& k, double dt, Cache<T> cache, const T* w,
                         const T* tmp, T* y, cudaStream_t s);

// krylov.cu
cudaError_t launch_reduce_partials(const double* partial, int nvec, int nparts, double* out,
                                   cudaStream_t s);
cudaError_t launch_sum_pair(const double* a, const double* b, const double* c, long long n,
                            double* partial, cudaStream_t s);
template <typename T>
cudaError_t launch_multi_dot(const T* V, long long ld, int nv, const T* w, long long n,
                             double* partial, cudaStream_t s);
template <typename T>
cudaError_t launch_cgs_update(const T* V, long long ld, int nv, const double* h, T* w,
                              long long n, int want_dots, double* partial, cudaStream_t s);
template <typename T>
cudaError_t launch_scale_from(const T* w, const double* alpha_dev, T* out, long long n,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_to_krylov(const double* x, double scale, T* out, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_lincomb(const T* V, long long ld, int nv, const double* y, T* out,
                           long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_axpy_to_double(double a, const T* x, double* y, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_residual_restart(const double* b, const T* Ax, double* r, long long n,
                                    double* partial, cudaStream_t s);
cudaError_t launch_norm2_double(const double* x, long long n, double* partial, cudaStream_t s);

// ras.cu
template <typename T>
cudaError_t launch_ras_factor(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off,
                              const T* J, T* coef, int threads, int ring_cells, size_t smem_bytes,
                              int* flags, cudaStream_t s);
template <typename T>
cudaError_t launch_ras_apply(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off,
                             const T* coef, const T* r, T* z, int ras_type, int threads,
                             const RasLaunch& L, T* gscratch, int* err, cudaStream_t s);

}  // namespace acac
