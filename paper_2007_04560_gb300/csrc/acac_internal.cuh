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
    double vol;          // hx*hy (*hz)
    float ihx2f, ihy2f;  // the same in float, for the FP32 Jacobian kernels
    int nz, dim;         // 3D: z extent (1 in 2D)
    double hz, ihz2;
    float ihz2f;
    // 1/(2 h^2) per axis: the weight of a face average (c_i + c_n) / 2 times a face
    // difference; no open-face test is needed with it, since a face at a Neumann wall has
    // the cell itself as neighbour and a zero difference
    double hihx2, hihy2, hihz2;
    float hihx2f, hihy2f, hihz2f;
    // 1 when every axis has the same spacing: a Laplacian then sums its neighbours first and
    // scales once by 1/h^2 (fewer FP64 operations than one scaling per axis)
    int iso;
};

// ---------------------------------------------------------------- 3D stencil
// 25 slots of the radius-2 stencil in 3D: 0 centre; 1..6 faces -x,+x,-y,+y,-z,+z;
// 7..12 two steps along an axis; 13..24 edge diagonals (xy, xz, yz).
constexpr int NSLOT3 = 25;
constexpr int CREC3 = 52;          // 3D record: 12 lower 2x2 blocks (+4 pad) | inverse pivot + 12 upper blocks
constexpr int NCOEF3 = 2 * CREC3;
__host__ __device__ constexpr int s3_dx(int s) {
    return (s == 1 || s == 13 || s == 15 || s == 17 || s == 19) ? -1 : (s == 2 || s == 14 || s == 16 || s == 18 || s == 20) ? 1
         : s == 7 ? -2 : s == 8 ? 2 : 0;
}
__host__ __device__ constexpr int s3_dy(int s) {
    return (s == 3 || s == 13 || s == 14 || s == 21 || s == 23) ? -1 : (s == 4 || s == 15 || s == 16 || s == 22 || s == 24) ? 1
         : s == 9 ? -2 : s == 10 ? 2 : 0;
}
__host__ __device__ constexpr int s3_dz(int s) {
    return (s == 5 || s == 17 || s == 18 || s == 21 || s == 22) ? -1 : (s == 6 || s == 19 || s == 20 || s == 23 || s == 24) ? 1
         : s == 11 ? -2 : s == 12 ? 2 : 0;
}
__host__ __device__ constexpr int slot3_of(int dx, int dy, int dz) {
    for (int s = 0; s < NSLOT3; ++s)
        if (s3_dx(s) == dx && s3_dy(s) == dy && s3_dz(s) == dz) return s;
    return -1;
}
// the 12 lower neighbours in increasing natural order (x fastest, then y, then z);
// the upper ones are their negatives in reverse order
__host__ __device__ constexpr int l3_dx(int k) { return (k == 2 || k == 7 || k == 11) ? -1 : (k == 4 || k == 9) ? 1 : k == 10 ? -2 : 0; }
__host__ __device__ constexpr int l3_dy(int k) { return (k == 1 || k == 7 || k == 8 || k == 9) ? -1 : k == 5 ? 1 : k == 6 ? -2 : 0; }
__host__ __device__ constexpr int l3_dz(int k) { return k == 0 ? -2 : (k >= 1 && k <= 5) ? -1 : 0; }
__host__ __device__ constexpr int u3_dx(int k) { return -l3_dx(11 - k); }
__host__ __device__ constexpr int u3_dy(int k) { return -l3_dy(11 - k); }
__host__ __device__ constexpr int u3_dz(int k) { return -l3_dz(11 - k); }
// faces in 3D: f = 0..5 is -x, +x, -y, +y, -z, +z
__host__ __device__ constexpr int f3_dx(int f) { return f == 0 ? -1 : f == 1 ? 1 : 0; }
__host__ __device__ constexpr int f3_dy(int f) { return f == 2 ? -1 : f == 3 ? 1 : 0; }
__host__ __device__ constexpr int f3_dz(int f) { return f == 4 ? -1 : f == 5 ? 1 : 0; }

__device__ __forceinline__ int wrap_or_clamp(int v, int n, bool periodic) {
    if (periodic) return v < 0 ? v + n : (v >= n ? v - n : v);
    return v < 0 ? 0 : (v >= n ? n - 1 : v);
}
// Neighbour index in 3D (wrapped or clamped per axis, as nb_index in 2D).
__device__ __forceinline__ int nb_index3(const Geom& g, int x, int y, int z, int dx, int dy, int dz) {
    const bool per = g.bc == ACAC_BC_PERIODIC;
    const int xx = wrap_or_clamp(x + dx, g.nx, per), yy = wrap_or_clamp(y + dy, g.ny, per);
    const int zz = wrap_or_clamp(z + dz, g.nz, per);
    return (zz * g.ny + yy) * g.nx + xx;
}
// 1/h^2 of face f of cell (x, y, z) if it carries flux, else 0.
template <typename T>
__device__ __forceinline__ T face_w3(const Geom& g, int x, int y, int z, int f) {
    const int xx = x + f3_dx(f), yy = y + f3_dy(f), zz = z + f3_dz(f);
    const bool open = g.bc == ACAC_BC_PERIODIC ||
                      (xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny && zz >= 0 && zz < g.nz);
    if (!open) return (T)0;
    if (sizeof(T) == 8) return (T)(f < 2 ? g.ihx2 : f < 4 ? g.ihy2 : g.ihz2);
    return (T)(f < 2 ? g.ihx2f : f < 4 ? g.ihy2f : g.ihz2f);
}

struct Coef {
    double alpha, beta, theta, gamma, rho;
    int S;
};

// ---------------------------------------------------------------- conversions
// Conversions between double and float, and from int to double, on the integer units: on
// this GPU a conversion instruction takes an FP64-pipe slot (it issues at the FP64
// multiply-add rate, 1/64 of the FP32 rate), and the FP64 pipe bounds the kernels that
// convert.  The results equal the conversion instructions' bit for bit (round to nearest
// even); operands whose result is not a normal number take the instruction.
__device__ __forceinline__ float dbl2flt(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long a = b & 0x7fffffffffffffffULL;
    // |x| in [2^-126, 2^128): exponent field 897..1150
    if (a - 0x3810000000000000ULL >= 0x0FE0000000000000ULL) return __double2float_rn(x);
    unsigned int f = (unsigned int)((a >> 29) - (896ULL << 23));    // rebiased exponent, top 23 bits
    const unsigned long long r = a & 0x1FFFFFFFULL;                  // the 29 bits dropped
    f += (unsigned int)((r > 0x10000000ULL) | ((r == 0x10000000ULL) & (f & 1u)));   // a carry may reach the exponent
    return __uint_as_float(f | ((unsigned int)(b >> 32) & 0x80000000u));
}
__device__ __forceinline__ double flt2dbl(float x) {
    const unsigned int b = __float_as_uint(x);
    const unsigned int a = b & 0x7fffffffu;
    if (a - 0x00800000u >= 0x7f000000u) return (double)x;            // zero, subnormal, inf, NaN
    const unsigned long long d = ((unsigned long long)a << 29) + (896ULL << 52);
    return __longlong_as_double((long long)(d | ((unsigned long long)(b & 0x80000000u) << 32)));
}
__device__ __forceinline__ double int2dbl(int i) {
    if (i == 0) return 0.0;
    const unsigned int a = i < 0 ? 0u - (unsigned int)i : (unsigned int)i;
    const int p = 31 - __clz(a);                                     // a in [2^p, 2^(p+1))
    const unsigned long long m = ((unsigned long long)a << (52 - p)) & 0x000FFFFFFFFFFFFFULL;
    const unsigned long long sgn = i < 0 ? 0x8000000000000000ULL : 0ULL;
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(1023 + p) << 52) | m));
}
// double -> Krylov precision T, and back
template <typename T>
__device__ __forceinline__ T from_dbl(double x) {
    if constexpr (sizeof(T) == 4) return dbl2flt(x);
    else return x;
}
template <typename T>
__device__ __forceinline__ double to_dbl(T x) {
    if constexpr (sizeof(T) == 4) return flt2dbl(x);
    else return x;
}

// ---------------------------------------------------------------- ensemble members
// An ensemble is `count` independent problems of one grid and one box decomposition,
// solved in lockstep: every launch covers all members, member m being a grid index
// (blockIdx.y of the cell, vector and box kernels, blockIdx.z of the 2D-tiled ones), and
// every per-member buffer holds `count` copies at a fixed stride (elements of the buffer's
// type).  A single problem is an ensemble of one (m = 0, strides unused).
struct MemberK {              // per-member scalars (device array)
    double alpha, beta, theta, gamma, rho;
    double dt;                // time step of the member's current attempt
    double lam;               // line-search step of the member's current trial
    double pad;
};
struct Members {
    int count = 1;
    const int* on = nullptr;      // on[m] == 0: member m sits the launch out (nullptr: all take part)
    const MemberK* k = nullptr;   // per-member scalars (nullptr: the launch's by-value scalars)
    long long vs = 0;             // 2N-vectors: states, residuals, directions, Krylov vectors
    long long gs = 0;             // 3-field buffers: G = [Gu | Gv | c], the product scratch
    long long cs = 0;             // linearisation cache (7 fields of N)
    long long js = 0;             // assembled stencil-diagonal Jacobian
    long long jps = 0;            // Jacobian records per box cell
    long long cfs = 0;            // Schwarz factors; 2x2 blocks of the fill solvers
    long long ss = 0;             // global scratch of the Schwarz apply (box vectors)
    long long rgs = 0;            // gathered right-hand side (windowed apply); fill solvers' inverse pivots
    long long zs = 0;             // box-cell results of the additive extensions (AS, right-RAS)
    long long ps = 0;             // reduction partials
    int rs = 0;                   // device scalars (reduction results, Hessenberg columns)
};
__device__ __forceinline__ bool member_off(const Members& mb, int m) { return mb.on && !mb.on[m]; }
// Coefficients of member m (the by-value ones when the launch has no per-member scalars).
__device__ __forceinline__ void member_coef(const Members& mb, int m, Coef& k) {
    if (!mb.k) return;
    const MemberK& q = mb.k[m];
    k.alpha = q.alpha;
    k.beta = q.beta;
    k.theta = q.theta;
    k.gamma = q.gamma;
    k.rho = q.rho;
}

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

// Dimension-generic cell helpers (faces 0..3 are -x, +x, -y, +y in both 2D and 3D).
template <int DIM>
__device__ __forceinline__ void decode_cell(const Geom& g, int c, int& x, int& y, int& z) {
    x = c % g.nx;
    if (DIM == 2) {
        y = c / g.nx;
        z = 0;
    } else {
        const int t = c / g.nx;
        y = t % g.ny;
        z = t / g.ny;
    }
}
template <int DIM>
__device__ __forceinline__ int face_nb(const Geom& g, int x, int y, int z, int f) {
    return DIM == 2 ? nb_index(g, x, y, face_dx(f), face_dy(f)) : nb_index3(g, x, y, z, f3_dx(f), f3_dy(f), f3_dz(f));
}
template <int DIM, typename T>
__device__ __forceinline__ T face_weight(const Geom& g, int x, int y, int z, int f) {
    return DIM == 2 ? face_w<T>(g, x, y, f) : face_w3<T>(g, x, y, z, f);
}
__device__ __forceinline__ double face_ih2(const Geom& g, int f) { return f < 2 ? g.ihx2 : f < 4 ? g.ihy2 : g.ihz2; }
template <typename T>
__device__ __forceinline__ T face_half(const Geom& g, int f) {
    if (sizeof(T) == 8) return (T)(f < 2 ? g.hihx2 : f < 4 ? g.hihy2 : g.hihz2);
    return (T)(f < 2 ? g.hihx2f : f < 4 ? g.hihy2f : g.hihz2f);
}
// Generic stencil slots (2D: 13, 3D: 25; slot f+1 is face f in both).
template <int DIM> __host__ __device__ constexpr int nslot() { return DIM == 2 ? NSLOT : NSLOT3; }
// boxes that can contain one grid cell (overlap below the owned box width): 2 per axis
template <int DIM> __host__ __device__ constexpr int rec_per_cell() { return DIM == 2 ? 4 : 8; }
template <int DIM> __host__ __device__ constexpr int sl_dx(int s) { return DIM == 2 ? slot_dx(s) : s3_dx(s); }
template <int DIM> __host__ __device__ constexpr int sl_dy(int s) { return DIM == 2 ? slot_dy(s) : s3_dy(s); }
template <int DIM> __host__ __device__ constexpr int sl_dz(int s) { return DIM == 2 ? 0 : s3_dz(s); }
template <int DIM> __host__ __device__ constexpr int sl_of(int dx, int dy, int dz) {
    return DIM == 2 ? (dz == 0 ? slot_of(dx, dy) : -1) : slot3_of(dx, dy, dz);
}
template <int DIM> __host__ __device__ constexpr int fc_dx(int f) { return DIM == 2 ? face_dx(f) : f3_dx(f); }
template <int DIM> __host__ __device__ constexpr int fc_dy(int f) { return DIM == 2 ? face_dy(f) : f3_dy(f); }
template <int DIM> __host__ __device__ constexpr int fc_dz(int f) { return DIM == 2 ? 0 : f3_dz(f); }
// face f of cell (x, y, z) is open: periodic, or its neighbour lies inside the grid
template <int DIM>
__device__ __forceinline__ bool face_open(const Geom& g, int x, int y, int z, int f) {
    if (g.bc == ACAC_BC_PERIODIC) return true;
    const int xx = x + fc_dx<DIM>(f), yy = y + fc_dy<DIM>(f), zz = z + fc_dz<DIM>(f);
    return xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny && (DIM == 2 || (zz >= 0 && zz < g.nz));
}
template <int DIM>
__device__ __forceinline__ int slot_nb(const Geom& g, int x, int y, int z, int s) {
    return DIM == 2 ? nb_index(g, x, y, slot_dx(s), slot_dy(s)) : nb_index3(g, x, y, z, s3_dx(s), s3_dy(s), s3_dz(s));
}

// Linearisation cache (Krylov precision T).  For cell k:
//   c, cu = dc/du1, cv = dc/dv1, Gu, Gv, du = dG_u/du1 pointwise part
//   (-alpha/2 + theta dphi/dp1 + theta dpsi/dq1), xc = theta (dphi/dp1 - dpsi/dq1).
//   dG_v/dv1 pointwise part = du + (alpha - beta)/2.
template <typename T>
struct Cache {
    T* c; T* cu; T* cv; T* Gu; T* Gv; T* du; T* xc;
};

// Scalars of the Jacobian in precision T, formed once on the host: a double division
// or conversion per thread runs on the FP64 pipe, which on sm_103 issues at 1/64 of
// the FP32 rate and would dominate the FP32 kernels.  The values are the correctly
// rounded ones a kernel would form.
// Member m's cache (the 7 fields at m * mb.cs).
template <typename T>
__device__ __forceinline__ Cache<T> member_cache(Cache<T> C, const Members& mb, int m) {
    const size_t o = (size_t)m * mb.cs;
    return Cache<T>{C.c + o, C.cu + o, C.cv + o, C.Gu + o, C.Gv + o, C.du + o, C.xc + o};
}

template <typename T>
struct JacK {
    T idt, irho, hg, dvs;   // 1/dt, 1/rho, gamma/2, (alpha - beta)/2
};
template <typename T>
inline JacK<T> jac_consts(const Coef& k, double dt) {
    return JacK<T>{(T)(1.0 / dt), (T)(1.0 / k.rho), (T)(0.5 * k.gamma), (T)(0.5 * (k.alpha - k.beta))};
}

// One subdomain of the Schwarz decomposition (Sec. 3.1).
struct SubInfo {
    int ox, oy;          // global coordinates of the box corner (may be < 0 when periodic)
    int W, H;            // box size
    int own_x0, own_x1;  // owned (non-overlapping) range, box-local
    int own_y0, own_y1;
    int oz, D;           // 3D: z corner and depth (0, 1 in 2D)
    int own_z0, own_z1;
    long long cell_base; // 3D: first entry in the level-ordered cell list / position map
    int nlev;            // wavefront levels = (W-1) + 2(H-1) + 1
    int lev_base;        // first entry of this subdomain in the level-offset table
    long long coef_base; // first coefficient of this subdomain
    long long vec_base;  // first padded-vector element in the global scratch
};

// Row pitch (in cells) of a padded box vector: W + 4, made odd so that the cells of
// one wavefront level (row stride pitch - 2) fall into distinct shared-memory banks.
__host__ __device__ constexpr int ras_pitch(int W) { return (W + 4) | 1; }
// The 3D row pitch: odd for doubles (fewer bank conflicts between the cells of a level,
// measured faster), W + 4 for floats (the larger vector then cost a CTA's stages: slower).
__host__ __device__ constexpr int ras3_pitch(int W, int value_bytes) { return value_bytes == 8 ? (W + 4) | 1 : W + 4; }

// Shared-memory plan of the Schwarz apply kernel (bytes / elements).
struct RasLaunch {
    int nbuf;            // coefficient stages in flight
    int threads;         // consumer warps (2 threads per cell of the widest level) + 1 producer warp
    int stage_elems;     // elements per stage (>= 28 x the largest level)
    int stage_off;       // byte offset of the stages (after mbarriers and level table)
    int vec_off;         // byte offset of the box vector (or of the level window) in shared memory
    size_t smem_bytes;   // dynamic shared memory per CTA
    int window;          // 1: windowed apply (last levels in shared memory, forward result in global)
    int win_cells;       // rows per window slot (the tallest box + 4)
    int stage_vec;       // windowed apply: element offset of the level's right-hand side in a stage
};

// Checks of acac_create (sizes, coefficients, partition, enumerations).
int validate_params(const acac_params* p);
// Grid sizes, spacings and the per-axis stencil weights of a validated parameter set.
Geom make_geom(const acac_params* p);

// 16 bytes of consecutive values as one vector word (bit casts, no aliasing)
__device__ __forceinline__ uint4 pack16(const float* p) {
    return make_uint4(__float_as_uint(p[0]), __float_as_uint(p[1]), __float_as_uint(p[2]), __float_as_uint(p[3]));
}
__device__ __forceinline__ uint4 pack16(const double* p) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(p[0]);
    const unsigned long long b = (unsigned long long)__double_as_longlong(p[1]);
    return make_uint4((unsigned)a, (unsigned)(a >> 32), (unsigned)b, (unsigned)(b >> 32));
}

// Deterministic two-stage reductions.  A reducing kernel runs at most RED_BLOCKS
// blocks of RED_THREADS threads (per ensemble member); each block writes one partial sum
// per reduced quantity v to partial[v * gridDim.x + block], and the block that finishes last
// adds the partials of each quantity in a fixed order (so the result does not
// depend on which block finishes when) and writes out[v].  The counter is zero
// between launches (the last block re-arms it); kernels that share one counter must
// not overlap in time (they are issued on one stream).
struct Red {
    double* partial;
    double* out;
    unsigned* counter;
};

// Member m's reduction: its partials, results and counter.
__device__ __forceinline__ Red member_red(Red r, const Members& mb, int m) {
    r.partial += (size_t)m * mb.ps;
    r.out += (size_t)m * mb.rs;
    r.counter += m;
    return r;
}

// Sum of v over the block (blockDim.x a multiple of 32), valid in thread 0.  sh: 32 doubles.
__device__ __forceinline__ double block_sum_red(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

// Grid of a reducing (or plain vector) kernel over n elements: about four elements per
// thread, at most RED_BLOCKS blocks.  Small problems (ensemble members) then leave
// most of the GPU to the kernels of other members instead of occupying every SM.
inline int red_grid(long long n) {
    const long long b = (n + 4LL * RED_THREADS - 1) / (4LL * RED_THREADS);
    return (int)(b < 1 ? 1 : (b > RED_BLOCKS ? RED_BLOCKS : b));
}

// Sum of v over the warp, valid in lane 0.
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Called by every thread of every block after the block's partials are written.  The
// last block sums up to eight quantities per pass: each warp adds its share of every
// quantity's partials and leaves one value per (quantity, warp) in shared memory, then
// one thread per quantity adds the warp values in order (two barriers per pass instead
// of two per quantity).
__device__ __forceinline__ void finish_reduction(const Red& r, int nv, double* sh) {
    (void)sh;
    __shared__ int s_last;
    __shared__ double s_w[8][32];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(r.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nb = gridDim.x;
    for (int v0 = 0; v0 < nv; v0 += 8) {
        const int c = nv - v0 < 8 ? nv - v0 : 8;
        for (int q = 0; q < c; ++q) {
            const double* p = r.partial + (size_t)(v0 + q) * nb;
            double a = 0.0;
            for (int i = threadIdx.x; i < nb; i += blockDim.x) a += __ldcg(p + i);
            a = warp_sum(a);
            if (lane == 0) s_w[q][warp] = a;
        }
        __syncthreads();
        if ((int)threadIdx.x < c) {
            double t = 0.0;
            for (int k = 0; k < nw; ++k) t += s_w[threadIdx.x][k];
            r.out[v0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *r.counter = 0u;
}

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
    Red red;             // ||F||^2 (one quantity)
    int* flags;          // bit 0: midpoint inadmissible, bit 1: trial state inadmissible
    const double* L0 = nullptr;   // discrete Laplacians of X0's two fields (launch_laplacian), or
                                  // null: formed from X0 in pass A
    const double* shift_sum = nullptr;   // if set, the trial shift is shift_sum[0] * shift_scale
    double shift_scale = 0.0;            // (read on the device: no host round trip)
    // pass A also writes the linearisation cache at the evaluated state (the state the next
    // Newton iteration linearises at when the line search accepts it): cache_mode 1 double
    // (cache_d), 2 float (cache_f), 0 none
    int cache_mode = 0;
    Cache<double> cache_d{};
    Cache<float> cache_f{};
    // 1: X is X0 itself (the first evaluation of a Newton solve, with L0 set): the midpoint is
    // the start state and sigma = 0, so pass A takes its shorter form (no series, no Laplacian
    // of X beyond 2 L0)
    int same = 0;
};
// Launchers take the members the launch covers last (default: a single problem).  Per
// member: X, X0, L0, Xt, S, F at stride vs; G at gs; the cache at cs; flags at 1; the
// reduction per member_red; shift_sum at rs; coefficients, dt and lam from mb.k.
cudaError_t launch_residual_g(const Geom& g, const Coef& k, const ResidualArgs& a, cudaStream_t s,
                              const Members& mb = Members{});
// L = discrete Laplacian of both fields of X (2N each): the start state's part of G3, fixed
// over a Newton solve
cudaError_t launch_laplacian(const Geom& g, const double* X, double* L, cudaStream_t s,
                             const Members& mb = Members{});
cudaError_t launch_residual_f(const Geom& g, const Coef& k, const ResidualArgs& a, cudaStream_t s,
                              const Members& mb = Members{});
cudaError_t launch_trial(const Geom& g, const ResidualArgs& a, cudaStream_t s, const Members& mb = Members{});
cudaError_t launch_table_log(const double* x, double* y, long long n, cudaStream_t s);
// energy and mass: two quantities
cudaError_t launch_energy(const Geom& g, const Coef& k, const double* X, Red red, int* flags, cudaStream_t s,
                          const Members& mb = Members{});
// wrt_x0 = 0: the cache of dF/dX1; 1: of dF/dX0 (the series derivative taken with -sigma;
// c, cu, cv, Gu, Gv are the same, and assembling with -dt gives the -1/dt diagonal).
template <typename T>
cudaError_t launch_linearize(const Geom& g, const Coef& k, const double* X, const double* X0,
                             const double* G, Cache<T> cache, cudaStream_t s, int wrt_x0 = 0);
// Adjoint: per-cell -mu^T dF/d(alpha, beta, theta, gamma) at (X1, X0) with G = [Gu | Gv | c]
// of pass A there, reduced to 4 sums (red.out[0..3]).
cudaError_t launch_param_grad(const Geom& g, const Coef& k, const double* X1, const double* X0,
                              const double* G, const double* mu, Red red, int* flags, cudaStream_t s);
// Loss L = wE E~(X) + wM/2 sum((u-u*)^2 + (v-v*)^2) dx dy: dL/dX into lam (2N) and the sums
// [L, dL/dalpha, dL/dbeta, dL/dtheta, dL/dgamma] into red.out[0..4].
cudaError_t launch_loss_grad(const Geom& g, const Coef& k, const double* X, const double* target, double wE,
                             double wM, double* lam, Red red, int* flags, cudaStream_t s);

// jacobian.cu
// The Jacobian kernels read their scalars (JacK, one per member) from device memory, written
// whenever dt or the coefficients change, so that a captured CUDA graph of a GMRES iteration
// stays valid across time steps.  Per member: J at js (records at jps), w, y at vs, the
// product scratch at gs, the cache at cs.
template <typename T>
cudaError_t launch_assemble(const Geom& g, const JacK<T>* kp, Cache<T> cache, T* J, cudaStream_t s,
                            const int* rec_of = nullptr, const Members& mb = Members{});
template <typename T>
cudaError_t launch_spmv(const Geom& g, const T* J, const T* w, T* y, cudaStream_t s, const Members& mb = Members{});
template <typename T>
cudaError_t launch_transpose(const Geom& g, const T* J, T* JT, cudaStream_t s);
template <typename T>
cudaError_t launch_jvp_tile(const Geom& g, const JacK<T>* kp, Cache<T> cache, const T* w, T* y, cudaStream_t s,
                            const Members& mb = Members{});
template <typename T>
cudaError_t launch_jvp_g(const Geom& g, const JacK<T>* kp, Cache<T> cache, const T* w, T* tmp,
                         cudaStream_t s, const Members& mb = Members{});
template <typename T>
cudaError_t launch_jvp_f(const Geom& g, const JacK<T>* kp, Cache<T> cache, const T* w, const T* tmp, T* y,
                         cudaStream_t s, const Members& mb = Members{});

// krylov.cu (per member: vectors at vs, device scalars at rs, the reduction per member_red)
cudaError_t launch_sum_pair(const double* a, const double* b, const double* c, long long n, Red red,
                            cudaStream_t s, const Members& mb = Members{});
template <typename T>
cudaError_t launch_multi_dot(const T* V, long long ld, int nv, const T* w, long long n, Red red,
                             cudaStream_t s, const Members& mb = Members{});
template <typename T>
cudaError_t launch_cgs_update(const T* V, long long ld, int nv, const double* h, T* w,
                              long long n, int want_norm, Red red, cudaStream_t s, const Members& mb = Members{});
template <typename T>
cudaError_t launch_scale_from(const T* w, const double* alpha_dev, T* out, long long n,
                              cudaStream_t s, const Members& mb = Members{});
// out = x * scale, or x * scale * (1 / scale_dev[m * sstride]) per member when scale_dev is set
template <typename T>
cudaError_t launch_to_krylov(const double* x, double scale, T* out, long long n, cudaStream_t s,
                             const Members& mb = Members{}, const double* scale_dev = nullptr, int sstride = 0);
// out = sum_{k < nv} y_k V_k, nv = nv_dev[m] per member when nv_dev is set
template <typename T>
cudaError_t launch_lincomb(const T* V, long long ld, int nv, const double* y, T* out,
                           long long n, cudaStream_t s, const Members& mb = Members{},
                           const int* nv_dev = nullptr);
template <typename T>
cudaError_t launch_axpy_to_double(double a, const T* x, double* y, long long n, cudaStream_t s,
                                  const Members& mb = Members{});
template <typename T>
cudaError_t launch_residual_restart(const double* b, double bsign, const T* Ax, double* r, long long n, Red red,
                                    cudaStream_t s, const Members& mb = Members{});
// ||a - b||^2 (b may be NULL)
cudaError_t launch_norm2_double(const double* a, const double* b, long long n, Red red, cudaStream_t s,
                                const Members& mb = Members{});
// y = x for the members that take part (vectors at vs)
cudaError_t launch_copy_members(const double* x, double* y, long long n, cudaStream_t s, const Members& mb);
// ensemble fields <-> member states: X[m] = [u[m] | v[m]] (to_state) or back
// X = [u | v] per member (u, v of member m at m * N) and, when Xp is set, ||X - Xp||^2 per
// member through red
cudaError_t launch_pack_state(const double* u, const double* v, double* X, const double* Xp, long long N, Red red,
                              cudaStream_t s, const Members& mb);
cudaError_t launch_pack_members(const double* u, const double* v, double* X, long long N, int to_state,
                                cudaStream_t s, const Members& mb);

// GMRES on the device (Sec. 3.1): the Givens rotations of the Hessenberg columns, the
// convergence test and the back substitution per member, so that a restart cycle needs
// no host read-back per Arnoldi step.
struct GmresHead {             // per member; written by the host at a cycle's start, read back after it
    double beta;               // ||r|| at the cycle's start
    double tol;                // absolute tolerance
    double resid;              // current residual estimate |g_{k}|
    int its, maxit;            // iterations so far (all cycles), limit
    int k;                     // Arnoldi steps of the current cycle
    int status;                // GMRES_RUNNING, GMRES_CONVERGED, GMRES_LIMIT, GMRES_NONFINITE
};
constexpr int GMRES_RUNNING = 0, GMRES_CONVERGED = 1, GMRES_LIMIT = 2, GMRES_NONFINITE = 3;
struct GmresWork {             // per member, device only
    double cs[MAX_RESTART], sn[MAX_RESTART], g[MAX_RESTART + 1];
    double R[MAX_RESTART * MAX_RESTART];   // rotated Hessenberg, column j at j * MAX_RESTART
};
// start of a cycle for the members with on[m]: g = beta e_1, k = 0 (gon[m] = on[m])
cudaError_t launch_gmres_start(GmresHead* head, GmresWork* work, const int* on, int* gon, int count,
                               cudaStream_t s);
// Arnoldi step j: column j = h0 + h1 (passes 2) or h0, subdiagonal sqrt(hn2), at red + m * rs
// (h0 at 0, h1 at MAX_RESTART + 1, hn2 at 2 (MAX_RESTART + 1)); updates the rotations, the
// residual estimate and gon[m] (0 once converged, at the limit or non-finite)
cudaError_t launch_gmres_givens(GmresHead* head, GmresWork* work, const double* red, int rs, int j, int passes,
                                int* gon, int count, cudaStream_t s);
// y = R^-1 g over the cycle's k steps into y + m * rs, k into kcnt[m] (members with on[m])
cudaError_t launch_gmres_solve(const GmresHead* head, const GmresWork* work, const int* on, double* y, int rs,
                               int* kcnt, int count, cudaStream_t s);

// ras.cu (per member: J at js or records at jps, factors at cfs, vectors at vs, scratch at
// ss, the gathered right-hand side at rgs, flags and err at 1)
// Jacobian rows of every box cell, one 4 x nslot-value record per box cell in the factor's
// order; rec_of[rec_per_cell * c + q] = the records of grid cell c (-1: unused).
template <typename T>
cudaError_t launch_repack(const Geom& g, const T* J, const int* rec_of, T* Jp, cudaStream_t s,
                          const Members& mb = Members{});
// J: stencil-diagonal (packed = 0) or the repacked records (packed = 1)
template <typename T>
cudaError_t launch_ras_factor(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off,
                              const T* J, int packed, T* coef, int threads, int ring_cells, size_t smem_bytes,
                              int* flags, cudaStream_t s, const Members& mb = Members{});
// ras_type AS / right-RAS: every box writes its cells' values by record into zb (2 values per
// box cell, member stride zs), then z is formed per grid cell from its records (rec_of) in a
// fixed order: launch_ext_gather.  Left-RAS writes the owned cells of z directly.
template <typename T>
cudaError_t launch_ras_apply(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off,
                             const T* coef, const T* r, T* z, int ras_type, int threads,
                             const RasLaunch& L, T* gscratch, const T* rg, int* err, cudaStream_t s,
                             const Members& mb = Members{}, const int* rec_of = nullptr, T* zb = nullptr);
template <typename T>
cudaError_t launch_ext_gather(const Geom& g, const int* rec_of, const T* zb, T* z, cudaStream_t s,
                              const Members& mb = Members{});
// 2D windowed apply: r restricted to every box cell (right-RAS: owned cells only), written by
// record (rec_of) into rg, two values per box cell
template <typename T>
cudaError_t launch_ras_gather(const Geom& g, const T* r, const int* rec_of, const unsigned char* own_of,
                              int ras_type, T* rg, cudaStream_t s, const Members& mb = Members{});

template <typename T>
cudaError_t launch_ras_factor3(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off, const int* cells,
                               const int* pos, const T* J, int packed, T* coef, int threads, int* flags,
                               cudaStream_t s, const Members& mb = Members{});
template <typename T>
cudaError_t launch_ras_apply3(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off, const int* cells,
                              const T* coef, const T* r, T* z, int ras_type, const RasLaunch& L, T* gscratch,
                              int* err, cudaStream_t s, const Members& mb = Members{}, const int* rec_of = nullptr,
                              T* zb = nullptr);

// Bounded wait for bit (word_bit) of a shared-memory word set by another warp of the block:
// true once set, false after limit_ns of the global timer (the caller then records an error
// and leaves instead of hanging).  One lane polls; the caller broadcasts the result.
__device__ __forceinline__ bool wait_bit_bounded(const volatile unsigned* word, int bit,
                                                 unsigned long long limit_ns) {
    if ((*word >> bit) & 1u) return true;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!((*word >> bit) & 1u)) {
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > limit_ns) return false;
        __nanosleep(128);
    }
    return true;
}
// The rows of the subdomain factorizations with fill wait at most this long for a row.
constexpr unsigned long long SPARSE_WAIT_NS = 2000000000ull;
// Self-check of the bounded waits (ras.cu): mode 0 an mbarrier phase that nothing completes,
// mode 1 a done bit that nothing sets; *status = ACAC_E_TIMEOUT when the wait gave up.
cudaError_t launch_wait_selftest(int mode, int* status, cudaStream_t s);

// subsolve.cu: subdomain solves with fill, ILU(1), ILU(2) and exact LU (Sec. 4.2, Table 2).
// The box matrix A_k is stored by 2x2 blocks on a pattern over the box's cells in natural
// order (x fastest); the pattern is that of the point factorization (the level of fill of
// a point entry is that of its cell pair, since every 2x2 block of A_k is full).
struct SparseShape {                 // host: symbolic factorization of one box shape
    int dim, W, H, D, n;             // box size, cells
    int band;                        // max |column - row| of the pattern (cells)
    int contig;                      // every row an interval of columns (the LU profile)
    std::vector<int> ptr, col, diag; // CSR of blocks, rows sorted; position of the pivot block
    std::vector<int> slot_pos;       // n x nslot: block of each stencil slot, -1 outside the box
    std::vector<int> flev_ptr, flev_rows;   // forward (L) dependency levels and their rows
    std::vector<int> blev_ptr, blev_rows;   // backward (U) dependency levels
};
// fill = 1 or 2: ILU(fill) by levels of fill; fill < 0: LU (every entry of the profile).
SparseShape build_sparse_shape(int dim, int W, int H, int D, int fill);

struct SparseShapeDev {              // device view of a SparseShape
    const int *ptr, *col, *diag, *slot_pos, *flev_ptr, *flev_rows, *blev_ptr, *blev_rows;
    int n, band, nflev, nblev, contig;
};
struct SparseBox {
    int shape;                       // index of its SparseShapeDev
    long long blk_base;              // first 2x2 block of the box in the value array
    long long cell_base;             // first cell of the box (pivot inverses, scratch vector)
};
// A_k of every box from the stencil-diagonal Jacobian J (values zeroed beforehand)
template <typename T>
cudaError_t launch_sparse_init(const Geom& g, int nbox, const SubInfo* subs, const SparseBox* boxes,
                               const SparseShapeDev* shapes, const T* J, T* val, cudaStream_t s,
                               const Members& mb = Members{});
// block IKJ factorization in place; D^-1 of every cell to dinv; bit 2 of *flags on a
// singular pivot block, bit 3 when a bounded wait for a row gave up.  smem: the done bits
// ((n + 31) / 32 words, rounded up to 4) and, with use_map, (threads / 32) x (2 band + 1)
// ints.
template <typename T>
cudaError_t launch_sparse_factor(int nbox, const SparseBox* boxes, const SparseShapeDev* shapes, T* val, T* dinv,
                                 int* flags, int threads, size_t smem, int use_map, cudaStream_t s,
                                 const Members& mb = Members{});
// z = sum_k E_k inv(L_k U_k) R_k r with the restrictions and extensions of ras_type; the
// box vector in shared memory (smem > 0) or in yscratch (2 values per box cell)
template <typename T>
cudaError_t launch_sparse_apply(const Geom& g, int nbox, const SubInfo* subs, const SparseBox* boxes,
                                const SparseShapeDev* shapes, const T* val, const T* dinv, const T* r, T* z,
                                int ras_type, T* yscratch, int threads, size_t smem, cudaStream_t s,
                                const Members& mb = Members{}, const int* rec_of = nullptr, T* zb = nullptr);

}  // namespace acac
