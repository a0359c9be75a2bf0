// Nonlinear residual F(X) of scheme (NSOA-1), its linearisation cache and the
// discrete energy / mass reductions.  All in FP64 (Sec. 2).
//
// The residual is computed in two passes so that the expensive per-cell work
// (two logarithms and the Lemma 2.2 series for p = u+v and q = u-v) is done exactly
// once per cell; the FP64 pipe, not HBM, bounds both passes on GB300:
//   pass A (g_kernel): G~^S = G1 + G2^S + G3 and the midpoint mobility c per cell;
//   pass B (f_kernel): F_u = (u1-u0)/dt - [div c~ grad G_u], F_v = (v1-v0)/dt + c G_v/rho,
//                      and per-block partial sums of ||F||^2.
#include <atomic>
#include <mutex>

#include <type_traits>

#include "acac_internal.cuh"

namespace acac {

__constant__ double c_taylor[MAX_S];   // 1 / ((2k)(2k+1)),  k = 1..S   (Lemma 2.2)
__constant__ double c_rcoef[MAX_S];    // 1 / (2k+1),        k = 1..S   (its sigma/zeta derivative)
__constant__ float c_rcoef_f[MAX_S];   // the same in float, for the FP32 Jacobian of the mixed form

// Table of the logarithm below: for F_j = 1 + j/1024, j = 0..1024, 1/F_j and ln F_j as an
// unevaluated sum hi + lo, one 32-byte entry per j.  Global memory read through the
// read-only cache: the lanes of a warp look up different j, which the constant cache would
// serve one address at a time.
constexpr int LOG_TABLE = 1025;
struct __align__(32) LogEntry {
    double inv, hi, lo, pad;
};
__device__ LogEntry d_log_tab[LOG_TABLE];

// The constant tables do not depend on S (S only selects how many terms a kernel
// sums), so they are uploaded once per device; several host threads may race here.
static std::mutex g_const_mu;
static std::atomic<unsigned long long> g_const_ready{0};   // bit d: device d holds the tables

cudaError_t set_taylor_constants(int) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ULL << (dev & 63);
    if (g_const_ready.load(std::memory_order_acquire) & bit) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_const_mu);
    if (g_const_ready.load(std::memory_order_relaxed) & bit) return cudaSuccess;
    std::vector<LogEntry> tab(LOG_TABLE);
    for (int j = 0; j < LOG_TABLE; ++j) {
        const long double F = 1.0L + (long double)j / 1024.0L;
        const long double L = logl(F);
        tab[j].inv = (double)(1.0L / F);
        tab[j].hi = (double)L;
        tab[j].lo = (double)(L - (long double)tab[j].hi);
        tab[j].pad = 0.0;
    }
    double a[MAX_S], b[MAX_S];
    float bf[MAX_S];
    for (int k = 1; k <= MAX_S; ++k) {
        a[k - 1] = 1.0 / ((2.0 * k) * (2.0 * k + 1.0));
        b[k - 1] = 1.0 / (2.0 * k + 1.0);
        bf[k - 1] = (float)b[k - 1];
    }
    e = cudaMemcpyToSymbol(d_log_tab, tab.data(), sizeof(LogEntry) * LOG_TABLE);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_taylor, a, sizeof(a));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rcoef, b, sizeof(b));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rcoef_f, bf, sizeof(bf));
    if (e == cudaSuccess) g_const_ready.fetch_or(bit, std::memory_order_release);
    return e;
}

// Natural logarithm in double by the table-driven reduction of P. T. P. Tang, "Table-
// driven implementation of the logarithm function in IEEE floating-point arithmetic"
// (ACM TOMS 16, 1990), written from the mathematics: x = 2^e m, m in [1, 2); F = 1 + j/1024
// is the table point nearest to m, so f = m - F is exact and |f| <= 2^-11; with
// u = f / F (one multiplication by the tabulated 1/F),
//     ln x = e ln 2 + ln F + ln(1 + u),
//     ln(1 + u) = u - u^2/2 + u^3/3 - u^4/4 + u^5/5 (the omitted terms are below 2^-57 |u|;
//     the larger table keeps the polynomial at five terms).
// ln 2 is split into a 42-bit head (so that e * head is exact) and a tail.  Arguments
// that are not positive normal numbers go to the library logarithm.  The GPU tests
// compare it with the library logarithm over the arguments the kernels use.  The range
// test and F are formed on the bit patterns (integer instructions): on this GPU every
// FP64 instruction costs an FP64-pipe slot, and those bound the kernels that call this.
// IEXP: the exponent's conversion to double on the integer units (int2dbl) or by the
// conversion instruction; the first is faster in every kernel measured but pass A with the
// FP64 cache (2.9% slower there).
template <bool IEXP = true>
__device__ __forceinline__ double table_log(double x) {
    const long long bits = __double_as_longlong(x);
    // positive normal numbers: bits in [bits(DBL_MIN), bits(DBL_MAX)]
    if ((unsigned long long)(bits - 0x0010000000000000LL) >= 0x7fe0000000000000ULL) return log(x);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    const long long mb = (bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL;
    const double m = __longlong_as_double(mb);
    const int j = (int)((mb >> 42) & 0x3ff) + (int)((mb >> 41) & 1);     // nearest j/1024
    const double F = __longlong_as_double(0x3ff0000000000000LL + ((long long)j << 42));   // 1 + j/1024
    const double2 t0 = __ldg(reinterpret_cast<const double2*>(&d_log_tab[j]));       // 1/F, ln F (hi)
    const double t1 = __ldg(&d_log_tab[j].lo);
    const double u = (m - F) * t0.x;
    const double u2 = u * u;
    // -1/2 + u (1/3 + u (-1/4 + u / 5))
    double q = fma(u, 0.2, -0.25);
    q = fma(u, q, 1.0 / 3.0);
    q = fma(u, q, -0.5);
    const double ln2_hi = 6.93147180559890330187045037746429443359375e-1;   // 42 significant bits
    const double ln2_lo = 5.497923018708371174712471233040e-14;
    const double ed = IEXP ? int2dbl(e) : (double)e;
    const double hi = fma(ed, ln2_hi, t0.y);
    const double lo = fma(ed, ln2_lo, t1);
    return hi + (u + fma(u2, q, lo));
}

// sum_{k=1..K} r^k / ((2k)(2k+1)), Horner form.
__device__ __forceinline__ double series_P(double r, int K) {
    double acc = c_taylor[K - 1];
    for (int k = K - 2; k >= 0; --k) acc = fma(acc, r, c_taylor[k]);
    return acc * r;
}

// Number of series terms K <= S, uniform over the warp, such that the terms K+1..S
// of every lane add up to less than 2^-60 of that lane's first term (the
// coefficients decrease, and r^K <= 2^-60 bounds the tail by a geometric series):
// the K-term sum then equals the S-term sum of Lemma 2.2 up to FP64 rounding.
// The same with a tail below 2^-bits (60 for double; 26 for the float Jacobian of the
// mixed form).  Every lane of the warp must call it.
__device__ __forceinline__ int series_terms_bits(float rmax_lane, int S, float bits) {
    // non-negative floats order like their bit patterns
    const unsigned ub = __float_as_uint(rmax_lane < 0.5f ? rmax_lane : 0.5f);
    const float r = __uint_as_float(__reduce_max_sync(0xffffffffu, ub));
    if (r <= 0.0f) return 1;
    if (r >= 0.25f) return S;
    // smallest K with r^K * (1 + r + r^2 + ...) <= 2^-bits, i.e. K >= (bits + log2(1/(1-r))) / log2(1/r)
    const int K = (int)ceilf((bits + 0.5f) / -log2f(r));
    return K < 1 ? 1 : (K > S ? S : K);
}
__device__ __forceinline__ int series_terms(double rmax_lane, int S) {
    return series_terms_bits(dbl2flt(rmax_lane), S, 60.0f);
}
// sum_{k=1..S} r^(k-1) / (2k+1), Horner form (in the precision T of the Jacobian).
template <typename T>
__device__ __forceinline__ T series_R(T r, int S);
template <>
__device__ __forceinline__ double series_R<double>(double r, int S) {
    double acc = c_rcoef[S - 1];
    for (int k = S - 2; k >= 0; --k) acc = fma(acc, r, c_rcoef[k]);
    return acc;
}
template <>
__device__ __forceinline__ float series_R<float>(float r, int S) {
    float acc = c_rcoef_f[S - 1];
    for (int k = S - 2; k >= 0; --k) acc = fmaf(acc, r, c_rcoef_f[k]);
    return acc;
}

// phi^S(zeta, sigma): series form of [Phi(zeta+sigma) - Phi(zeta-sigma)] / (2 sigma)
// (Lemma 2.2, Eq. D2-1, combination f_S(zeta,sigma) - f_S(1-zeta,sigma)):
//   ln(zeta/(1-zeta)) - sum_k [(sigma/zeta)^{2k} - (sigma/(1-zeta))^{2k}] / ((2k)(2k+1)).
// The squares ra = (sigma/zeta)^2, rb = (sigma/(1-zeta))^2 and the log argument are
// formed first (series_args2) so that the caller can pick the warp-uniform term count.
struct SeriesArgs {
    double ra, rb, ratio;
    double a, b;     // sigma / zeta, sigma / (1 - zeta)
    double iz, io;   // 1 / zeta, 1 / (1 - zeta) divided by the common factor of the inputs
};
template <bool IEXP = true>
__device__ __forceinline__ double phi_series(const SeriesArgs& s, int K) {
    return table_log<IEXP>(s.ratio) - (series_P(s.ra, K) - series_P(s.rb, K));
}

// 1 - (u + v) and 1 - (u - v), each correctly rounded from the doubles u, v: 1 - u is split
// into its rounded value s and the rounding error e (s + e = 1 - u exactly, the two-sum of
// 1 and -u), and s -+ v is exact wherever the result is small (s and v then lie within a
// factor 2 of each other), so only the final addition of e rounds.
__device__ __forceinline__ void one_minus_pq(double u, double v, double& mp, double& mq) {
    const double s = 1.0 - u;
    const double e = -u - (s - 1.0);
    mp = (s - v) + e;
    mq = (s + v) + e;
}

// Twice the midpoints zeta, 1 - zeta and half-increments sigma of p = u + v and q = u - v
// (Eq. D2-1), formed from the end states so that each keeps its relative accuracy near a
// pure phase: zeta from p1 + p0 (each sum of u and v rounds relative to its own, possibly
// tiny, value), 1 - zeta from the end values 1 - p, 1 - q (one_minus_pq), sigma from the
// differences of whichever end values lie nearer zero.  Subtracting a rounded zeta from 1, or summing u1 + u0 and v1 + v0 before adding
// them, leaves an absolute error of ~1e-16 that swamps zeta or 1 - zeta once either falls
// towards 1e-8.
struct Midpoint2 {
    double zp, omp, sp, zq, omq, sq;
};
// true unless 0 < x2 / 2 < 1 keeps at least 2^-6 from both ends (x2 = twice a midpoint; the
// bit pattern of a positive double orders like its value, a negative one or NaN falls outside)
__device__ __forceinline__ bool near_pure2(double x2) {
    const long long b = __double_as_longlong(x2);
    return b < 0x3FA0000000000000LL || b > 0x3FFF800000000000LL;   // 2^-5, 2 - 2^-5
}
__device__ __forceinline__ Midpoint2 midpoint_pq2(double u1, double v1, double u0, double v0) {
    const double p1 = u1 + v1, p0 = u0 + v0, q1 = u1 - v1, q0 = u0 - v0;
    double mp1, mq1, mp0, mq0;
    one_minus_pq(u1, v1, mp1, mq1);
    one_minus_pq(u0, v0, mp0, mq0);
    const double zp = p1 + p0, zq = q1 + q0;
    // sigma from the end values nearer zero: p1 - p0 below zeta = 1/2, (1-p0) - (1-p1) above
    return Midpoint2{zp, mp1 + mp0, zp < 1.0 ? p1 - p0 : mp0 - mp1,
                     zq, mq1 + mq0, zq < 1.0 ? q1 - q0 : mq0 - mq1};
}

// The same quantities at the cost of the plain sums: 2 zeta = (u1 + u0) +- (v1 + v0),
// 2 (1 - zeta) = 2 - 2 zeta, 2 sigma = (u1 - u0) +- (v1 - v0).  Far from a pure phase these
// carry errors of a few units in the last place of u and v, i.e. of zeta and 1 - zeta (both
// >= 2^-6 there); when a lane of the warp comes within 2^-6 of a pure phase the whole warp
// takes midpoint_pq2 instead (one vote per warp; every lane of the warp must call it).
__device__ __forceinline__ Midpoint2 midpoint_pq2_fast(double u1, double v1, double u0, double v0) {
    const double su = u1 + u0, sv = v1 + v0, du = u1 - u0, dv = v1 - v0;
    Midpoint2 m{su + sv, 0.0, du + dv, su - sv, 0.0, du - dv};
    m.omp = 2.0 - m.zp;
    m.omq = 2.0 - m.zq;
    if (__any_sync(0xffffffffu, near_pure2(m.zp) || near_pure2(m.zq))) m = midpoint_pq2(u1, v1, u0, v0);
    return m;
}
// midpoint_pq2_fast for equal end states (u1 = u0 = u, v1 = v0 = v): the same values,
// sigma = +0, without the differences
__device__ __forceinline__ Midpoint2 midpoint_pq2_same(double u, double v) {
    const double su = u + u, sv = v + v;
    Midpoint2 m{su + sv, 0.0, 0.0, su - sv, 0.0, 0.0};
    m.omp = 2.0 - m.zp;
    m.omq = 2.0 - m.zq;
    if (__any_sync(0xffffffffu, near_pure2(m.zp) || near_pure2(m.zq))) m = midpoint_pq2(u, v, u, v);
    return m;
}
// positive and finite (bit-pattern test, no floating-point compare)
__device__ __forceinline__ bool pos_bits(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7FF0000000000000LL;
}

// series_args for p and q with one division: 1/(zp(1-zp)) and 1/(zq(1-zq)) from the
// reciprocal of their product (which stays far above the underflow threshold for any
// state that is not within 1e-140 of a pure phase; such states take two divisions).
// zeta, 1 - zeta and sigma come in separately (see midpoint_pq) and may all carry the
// same positive factor: the ratios sigma/zeta, sigma/(1-zeta), zeta/(1-zeta) do not see it.
__device__ __forceinline__ void series_args2(double zp, double omp, double sp, double zq, double omq, double sq,
                                             SeriesArgs& ap, SeriesArgs& aq) {
    const double Pp = zp * omp, Pq = zq * omq;
    const double PP = Pp * Pq;
    double invp, invq;
    // PP > 1e-280 on the bit patterns (PP >= 0 here: the callers pass positive midpoints)
    if (__double_as_longlong(PP) > __double_as_longlong(1e-280)) {
        const double D = 1.0 / PP;
        invp = Pq * D;
        invq = Pp * D;
    } else {
        invp = 1.0 / Pp;
        invq = 1.0 / Pq;
    }
    const double tp = zp * invp, up = omp * invp;      // 1/(1-zp), 1/zp
    const double tq = zq * invq, uq = omq * invq;
    const double a1 = sp * up, b1 = sp * tp, a2 = sq * uq, b2 = sq * tq;
    ap = SeriesArgs{a1 * a1, b1 * b1, zp * tp, a1, b1, up, tp};
    aq = SeriesArgs{a2 * a2, b2 * b2, zq * tq, a2, b2, uq, tq};
}

// series_args2 for sigma = 0: the series arguments vanish and only the log argument and the
// reciprocals remain (the values series_args2 gives for sp = sq = +0)
__device__ __forceinline__ void series_args2_same(double zp, double omp, double zq, double omq, SeriesArgs& ap,
                                                  SeriesArgs& aq) {
    const double Pp = zp * omp, Pq = zq * omq;
    const double PP = Pp * Pq;
    double invp, invq;
    if (__double_as_longlong(PP) > __double_as_longlong(1e-280)) {
        const double D = 1.0 / PP;
        invp = Pq * D;
        invq = Pp * D;
    } else {
        invp = 1.0 / Pp;
        invq = 1.0 / Pq;
    }
    const double tp = zp * invp, up = omp * invp;
    const double tq = zq * invq, uq = omq * invq;
    ap = SeriesArgs{0.0, 0.0, zp * tp, 0.0, 0.0, up, tp};
    aq = SeriesArgs{0.0, 0.0, zq * tq, 0.0, 0.0, uq, tq};
}

// max of non-negative doubles (their bit patterns order like the values)
__device__ __forceinline__ double max_nonneg(double a, double b, double c, double d) {
    long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    const long long z = __double_as_longlong(c), w = __double_as_longlong(d);
    x = x > y ? x : y;
    x = x > z ? x : z;
    return __longlong_as_double(x > w ? x : w);
}

// d phi^S / d(end value) where zeta and sigma both move by 1/2, for p and q at once:
//   1/2 [ (1 + a^2 R(a^2) - a R(a^2)) / zeta + (1 + b^2 R(b^2) + b R(b^2)) / (1 - zeta) ],
// a = sigma/zeta, b = sigma/(1-zeta), in the Jacobian's precision T.  The four
// reciprocals come from one division; in double R is summed to a warp-uniform K terms
// whose omitted tail is below 2^-60 of its first term (every lane of the warp must call
// it), in float to all S terms.
template <typename T>
__device__ __forceinline__ void dphi_pair(T zp, T omp, T sp, T zq, T omq, T sq, int S, T& dp, T& dq) {
    const T Pp = zp * omp, Pq = zq * omq, PP = Pp * Pq;
    T invp, invq;
    if (PP > (sizeof(T) == 8 ? (T)1e-280 : (T)1e-30)) {
        const T D = (T)1 / PP;
        invp = Pq * D;
        invq = Pp * D;
    } else {
        invp = (T)1 / Pp;
        invq = (T)1 / Pq;
    }
    const T izp = omp * invp, iop = zp * invp, izq = omq * invq, ioq = zq * invq;
    const T a1 = sp * izp, b1 = sp * iop, a2 = sq * izq, b2 = sq * ioq;
    const T ra1 = a1 * a1, rb1 = b1 * b1, ra2 = a2 * a2, rb2 = b2 * b2;
    // FP32 sums all S terms: its FMAs cost less than the vote
    const int K = sizeof(T) == 8 ? series_terms_bits((float)max_nonneg((double)ra1, (double)rb1, (double)ra2,
                                                                       (double)rb2), S, 60.0f)
                                 : S;
    const T R1 = series_R<T>(ra1, K), R2 = series_R<T>(rb1, K), R3 = series_R<T>(ra2, K), R4 = series_R<T>(rb2, K);
    const T one = (T)1, half = (T)0.5;
    dp = half * ((one + ra1 * R1 - a1 * R1) * izp + (one + rb1 * R2 + b1 * R2) * iop);
    dq = half * ((one + ra2 * R3 - a2 * R3) * izq + (one + rb2 * R4 + b2 * R4) * ioq);
}

// ---------------------------------------------------------------- pass A
// x in (0, 1) on the IEEE bit pattern: positive doubles order like their bits, and
// every negative number, NaN or value >= 1 falls outside (0, bits(1.0)).
__device__ __forceinline__ bool in_unit(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x3ff0000000000000LL;
}

// d phi^S / d(end value) from the series arguments of pass A: dphi_pair's
//   1/2 [(1 + a^2 R(a^2) - a R(a^2)) / zeta + (1 + b^2 R(b^2) + b R(b^2)) / (1 - zeta)],
// where pass A's inputs were doubled, so that iz = 1/(2 zeta) and io = 1/(2 (1 - zeta)) already
// carry the 1/2; in double with pass A's warp-uniform K terms, or in float with all S terms.
template <typename T>
__device__ __forceinline__ T dphi_from_args(const SeriesArgs& s, int K) {
    const T a = from_dbl<T>(s.a), b = from_dbl<T>(s.b), ra = from_dbl<T>(s.ra), rb = from_dbl<T>(s.rb);
    const T R1 = series_R<T>(ra, K), R2 = series_R<T>(rb, K);
    const T one = (T)1;
    return (one + ra * R1 - a * R1) * from_dbl<T>(s.iz) + (one + rb * R2 + b * R2) * from_dbl<T>(s.io);
}

// SAME (with PRE): X is X0 itself, so u1 = u0, the Laplacian of X1 + X0 is 2 L0, sigma = 0
// and phi^S = ln(zeta / (1 - zeta)) (the series of K = 1 terms at sigma = 0 adds exactly 0).
// Three blocks per SM: without a minimum the compiler held the float-cache form to 64
// registers with a spill; at 78 registers (24 resident warps, enough for the FP64 pipe) its
// trial evaluations run 4% faster.
template <int DIM, bool PRE, int CM, bool SAME = false>
__global__ void __launch_bounds__(256, 3) g_kernel(Geom g, Coef k, ResidualArgs a, Members mb) {
    const int N = g.N;
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    member_coef(mb, m, k);
    a.X += (size_t)m * mb.vs;
    a.X0 += (size_t)m * mb.vs;
    if (PRE) a.L0 += (size_t)m * mb.vs;
    a.G += (size_t)m * mb.gs;
    a.flags += m;
    if (CM == 1) {
        const size_t o = (size_t)m * mb.cs;
        a.cache_d = Cache<double>{a.cache_d.c + o, a.cache_d.cu + o, a.cache_d.cv + o, a.cache_d.Gu + o,
                                  a.cache_d.Gv + o, a.cache_d.du + o, a.cache_d.xc + o};
    } else if (CM == 2) {
        const size_t o = (size_t)m * mb.cs;
        a.cache_f = Cache<float>{a.cache_f.c + o, a.cache_f.cu + o, a.cache_f.cv + o, a.cache_f.Gu + o,
                                 a.cache_f.Gv + o, a.cache_f.du + o, a.cache_f.xc + o};
    }
    const double* __restrict__ Xu = a.X;
    const double* __restrict__ Xv = a.X + N;
    const double* __restrict__ Pu = a.X0;
    const double* __restrict__ Pv = a.X0 + N;
    int flag = 0;
    // uniform trip count so that every lane of a warp takes part in the term-count vote
    const int stride = gridDim.x * blockDim.x;
    const int iters = (N + stride - 1) / stride;
    for (int it = 0; it < iters; ++it) {
        const int c = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const bool live = c < N;
        const int cc = live ? c : N - 1;
        int x, y, z;
        decode_cell<DIM>(g, cc, x, y, z);
        const double u1 = Xu[cc], v1 = Xv[cc], u0 = SAME ? u1 : Pu[cc], v0 = SAME ? v1 : Pv[cc];
        const double su = u1 + u0, sv = v1 + v0;
        // Laplacians of u1 + u0 and v1 + v0 (G3), per axis (S_- + S_+ - 2 S) / h^2; a
        // clamped (Neumann ghost) neighbour is the cell itself and adds nothing.  With PRE
        // the start state's Laplacians come precomputed (fixed over a Newton solve)
        double lu = 0.0, lv = 0.0;
        if (SAME) {
            lu = 2.0 * a.L0[cc];
            lv = 2.0 * a.L0[N + cc];
        } else if (g.iso) {
            // equal spacing: the neighbour sums first, one scaling by 1/h^2 (with PRE the
            // start state's Laplacians enter as the addend of that scaling)
            double nu = 0.0, nv = 0.0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const int nm = face_nb<DIM>(g, x, y, z, 2 * d), np = face_nb<DIM>(g, x, y, z, 2 * d + 1);
                const double tu = PRE ? Xu[nm] + Xu[np] : (Xu[nm] + Pu[nm]) + (Xu[np] + Pu[np]);
                const double tv = PRE ? Xv[nm] + Xv[np] : (Xv[nm] + Pv[nm]) + (Xv[np] + Pv[np]);
                nu = d == 0 ? tu : nu + tu;
                nv = d == 0 ? tv : nv + tv;
            }
            const double c2 = -2.0 * DIM, ih2 = g.ihx2;
            if (PRE) {
                lu = fma(fma(c2, u1, nu), ih2, a.L0[cc]);
                lv = fma(fma(c2, v1, nv), ih2, a.L0[N + cc]);
            } else {
                lu = fma(c2, su, nu) * ih2;
                lv = fma(c2, sv, nv) * ih2;
            }
        } else {
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const double ih2 = face_ih2(g, 2 * d);
                const int nm = face_nb<DIM>(g, x, y, z, 2 * d), np = face_nb<DIM>(g, x, y, z, 2 * d + 1);
                if (PRE) {
                    lu = fma(fma(-2.0, u1, Xu[nm] + Xu[np]), ih2, lu);
                    lv = fma(fma(-2.0, v1, Xv[nm] + Xv[np]), ih2, lv);
                } else {
                    lu = fma(fma(-2.0, su, (Xu[nm] + Pu[nm]) + (Xu[np] + Pu[np])), ih2, lu);
                    lv = fma(fma(-2.0, sv, (Xv[nm] + Pv[nm]) + (Xv[np] + Pv[np])), ih2, lv);
                }
            }
            if (PRE) {
                lu += a.L0[cc];
                lv += a.L0[N + cc];
            }
        }
        // G2^S on p = u+v and q = u-v at the midpoint (zeta) with half-increment (sigma),
        // all three doubled (the series only sees their ratios)
        const Midpoint2 m2 = SAME ? midpoint_pq2_same(u1, v1) : midpoint_pq2_fast(u1, v1, u0, v0);
        const bool ok = pos_bits(m2.zp) && pos_bits(m2.omp) && pos_bits(m2.zq) && pos_bits(m2.omq);
        if (live && !ok) flag |= 1;
        SeriesArgs ap, aq;
        int K = 1;
        double phi, psi;
        if (SAME) {
            series_args2_same(ok ? m2.zp : 1.0, ok ? m2.omp : 1.0, ok ? m2.zq : 1.0, ok ? m2.omq : 1.0, ap, aq);
            phi = table_log<CM != 1>(ap.ratio);
            psi = table_log<CM != 1>(aq.ratio);
        } else {
            series_args2(ok ? m2.zp : 1.0, ok ? m2.omp : 1.0, m2.sp, ok ? m2.zq : 1.0, ok ? m2.omq : 1.0, m2.sq,
                         ap, aq);
            K = series_terms(max_nonneg(ap.ra, ap.rb, aq.ra, aq.rb), k.S);
            phi = phi_series<CM != 1>(ap, K);
            psi = phi_series<CM != 1>(aq, K);
        }
        if (!ok) { phi = 0.0; psi = 0.0; }
        const double ha = 0.5 * k.alpha, hgn = -0.5 * k.gamma;
        const double Gu = fma(hgn, lu, fma(k.theta, phi + psi, fma(-ha, su, ha)));
        const double Gv = fma(hgn, lv, fma(k.theta, phi - psi, -0.5 * k.beta * sv));
        const double ub = 0.5 * su, vb = 0.5 * sv;
        const double cmob = ub * (1.0 - ub) * (0.25 - vb * vb);
        if (live) {
            a.G[c] = Gu;
            a.G[N + c] = Gv;
            a.G[2 * N + c] = cmob;
        }
        if (CM != 0) {
            // the linearisation cache at this state (linearize_kernel's entries, same formulas)
            using T = typename std::conditional<CM == 1, double, float>::type;
            const int KT = CM == 1 ? K : k.S;
            // sigma = 0: both series factors are exactly 1, the derivative is 1/zeta + 1/(1-zeta)
            // (halved through the doubled inputs)
            const T dp = SAME ? from_dbl<T>(ap.iz) + from_dbl<T>(ap.io) : dphi_from_args<T>(ap, KT);
            const T dq = SAME ? from_dbl<T>(aq.iz) + from_dbl<T>(aq.io) : dphi_from_args<T>(aq, KT);
            if (live) {
                Cache<T> C;
                if constexpr (CM == 1) C = a.cache_d; else C = a.cache_f;
                const T theta = from_dbl<T>(k.theta), halpha = from_dbl<T>(0.5 * k.alpha);
                const T A = theta * dp, B = theta * dq;
                const T ubT = from_dbl<T>(ub), vbT = from_dbl<T>(vb);
                C.c[c] = from_dbl<T>(cmob);
                C.cu[c] = (T)0.5 * ((T)1 - (T)2 * ubT) * ((T)0.25 - vbT * vbT);
                C.cv[c] = -ubT * ((T)1 - ubT) * vbT;
                C.Gu[c] = from_dbl<T>(Gu);
                C.Gv[c] = from_dbl<T>(Gv);
                C.du[c] = -halpha + A + B;
                C.xc[c] = A - B;
            }
        }
    }
    if (flag) atomicOr(a.flags, flag);
}

// Trial state of the line search: Xt_u = X_u + lam (S_u + shift), Xt_v = X_v + lam S_v,
// with flag bit 1 when some u+v or u-v leaves (0, 1).
__global__ void __launch_bounds__(256) trial_kernel(int N, ResidualArgs a, Members mb) {
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    a.X += (size_t)m * mb.vs;
    a.S += (size_t)m * mb.vs;
    a.Xt += (size_t)m * mb.vs;
    a.flags += m;
    if (mb.k) a.lam = mb.k[m].lam;
    int flag = 0;
    const double shift = a.shift_sum ? a.shift_sum[(size_t)m * mb.rs] * a.shift_scale : a.shift;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const double u = fma(a.lam, a.S[c] + shift, a.X[c]);
        const double v = fma(a.lam, a.S[N + c], a.X[N + c]);
        a.Xt[c] = u;
        a.Xt[N + c] = v;
        if (!(in_unit(u + v) && in_unit(u - v))) flag |= 2;
    }
    if (flag) atomicOr(a.flags, flag);
}

// ---------------------------------------------------------------- pass B
template <int DIM>
__global__ void __launch_bounds__(256) f_kernel(Geom g, double idt, double irho, ResidualArgs a, Members mb) {
    __shared__ double sh[32];
    const int N = g.N;
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    if (mb.k) {
        // correctly rounded, as the host forms them for the by-value arguments
        idt = 1.0 / mb.k[m].dt;
        irho = 1.0 / mb.k[m].rho;
    }
    a.X += (size_t)m * mb.vs;
    a.X0 += (size_t)m * mb.vs;
    a.G += (size_t)m * mb.gs;
    a.F += (size_t)m * mb.vs;
    a.red = member_red(a.red, mb, m);
    const double* __restrict__ X1 = a.X;
    const double* __restrict__ Gu = a.G;
    const double* __restrict__ Gv = a.G + N;
    const double* __restrict__ cm = a.G + 2 * N;
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int x, y, z;
        decode_cell<DIM>(g, c, x, y, z);
        const double gc = Gu[c], cc = cm[c];
        // the faces of an axis (of every axis, with equal spacing) share the weight 1/(2 h^2),
        // applied once to their sum (a Neumann wall's neighbour is the cell itself: its
        // difference is exactly zero)
        double div = 0.0;
        if (g.iso) {
            double t = 0.0;
#pragma unroll
            for (int f = 0; f < 2 * DIM; ++f) {
                const int n = face_nb<DIM>(g, x, y, z, f);
                t = f == 0 ? (cc + cm[n]) * (Gu[n] - gc) : fma(cc + cm[n], Gu[n] - gc, t);
            }
            div = g.hihx2 * t;
        } else {
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const int nm = face_nb<DIM>(g, x, y, z, 2 * d), np = face_nb<DIM>(g, x, y, z, 2 * d + 1);
                const double t = fma(cc + cm[np], Gu[np] - gc, (cc + cm[nm]) * (Gu[nm] - gc));
                div = fma(face_half<double>(g, 2 * d), t, div);
            }
        }
        const double Fu = (X1[c] - a.X0[c]) * idt - div;
        const double Fv = (X1[N + c] - a.X0[N + c]) * idt + cc * Gv[c] * irho;
        a.F[c] = Fu;
        a.F[N + c] = Fv;
        acc = fma(Fu, Fu, fma(Fv, Fv, acc));
    }
    const double t = block_sum_red(acc, sh);
    if (threadIdx.x == 0) a.red.partial[blockIdx.x] = t;
    finish_reduction(a.red, 1, sh);
}

static int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < RED_BLOCKS ? (b < 1 ? 1 : b) : RED_BLOCKS);
}

cudaError_t launch_residual_g(const Geom& g, const Coef& k, const ResidualArgs& a, cudaStream_t s,
                              const Members& mb) {
    cudaError_t e = set_taylor_constants(k.S);
    if (e != cudaSuccess) return e;
    const int nb = grid_for(g.N, 256);
    auto go = [&](auto dimc, auto prec, auto cmc) {
        constexpr int D = decltype(dimc)::value, C = decltype(cmc)::value;
        constexpr bool P = decltype(prec)::value;
        if constexpr (P) {
            if (a.same) {
                g_kernel<D, true, C, true><<<dim3(nb, mb.count), 256, 0, s>>>(g, k, a, mb);
                return;
            }
        }
        g_kernel<D, P, C, false><<<dim3(nb, mb.count), 256, 0, s>>>(g, k, a, mb);
    };
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using PT = std::true_type;
    using PF = std::false_type;
    using C0 = std::integral_constant<int, 0>;
    using C1 = std::integral_constant<int, 1>;
    using C2 = std::integral_constant<int, 2>;
    if (g.dim == 3) {
        if (a.L0) {
            if (a.cache_mode == 1) go(I3{}, PT{}, C1{}); else if (a.cache_mode == 2) go(I3{}, PT{}, C2{}); else go(I3{}, PT{}, C0{});
        } else {
            go(I3{}, PF{}, C0{});
        }
    } else {
        if (a.L0) {
            if (a.cache_mode == 1) go(I2{}, PT{}, C1{}); else if (a.cache_mode == 2) go(I2{}, PT{}, C2{}); else go(I2{}, PT{}, C0{});
        } else {
            go(I2{}, PF{}, C0{});
        }
    }
    return cudaGetLastError();
}

template <int DIM>
__global__ void __launch_bounds__(256) laplacian_kernel(Geom g, const double* __restrict__ X, double* __restrict__ L,
                                                        Members mb) {
    const int N = g.N;
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    X += (size_t)m * mb.vs;
    L += (size_t)m * mb.vs;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int x, y, z;
        decode_cell<DIM>(g, c, x, y, z);
        const double u = X[c], v = X[N + c];
        double lu = 0.0, lv = 0.0;
        if (g.iso) {
            double nu = 0.0, nv = 0.0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const int nm = face_nb<DIM>(g, x, y, z, 2 * d), np = face_nb<DIM>(g, x, y, z, 2 * d + 1);
                nu = d == 0 ? X[nm] + X[np] : nu + (X[nm] + X[np]);
                nv = d == 0 ? X[N + nm] + X[N + np] : nv + (X[N + nm] + X[N + np]);
            }
            lu = fma(-2.0 * DIM, u, nu) * g.ihx2;
            lv = fma(-2.0 * DIM, v, nv) * g.ihx2;
        } else {
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const double ih2 = face_ih2(g, 2 * d);
                const int nm = face_nb<DIM>(g, x, y, z, 2 * d), np = face_nb<DIM>(g, x, y, z, 2 * d + 1);
                lu = fma(fma(-2.0, u, X[nm] + X[np]), ih2, lu);
                lv = fma(fma(-2.0, v, X[N + nm] + X[N + np]), ih2, lv);
            }
        }
        L[c] = lu;
        L[N + c] = lv;
    }
}

cudaError_t launch_laplacian(const Geom& g, const double* X, double* L, cudaStream_t s, const Members& mb) {
    const dim3 nb(grid_for(g.N, 256), mb.count);
    if (g.dim == 3) laplacian_kernel<3><<<nb, 256, 0, s>>>(g, X, L, mb);
    else laplacian_kernel<2><<<nb, 256, 0, s>>>(g, X, L, mb);
    return cudaGetLastError();
}

cudaError_t launch_trial(const Geom& g, const ResidualArgs& a, cudaStream_t s, const Members& mb) {
    trial_kernel<<<dim3(grid_for(g.N, 256), mb.count), 256, 0, s>>>(g.N, a, mb);
    return cudaGetLastError();
}

cudaError_t launch_residual_f(const Geom& g, const Coef& k, const ResidualArgs& a, cudaStream_t s,
                              const Members& mb) {
    // 1/dt and 1/rho on the host (correctly rounded, as a kernel division would be)
    const double idt = 1.0 / a.dt, irho = 1.0 / k.rho;
    const dim3 nb(red_grid(g.N), mb.count);
    if (g.dim == 3) f_kernel<3><<<nb, RED_THREADS, 0, s>>>(g, idt, irho, a, mb);
    else f_kernel<2><<<nb, RED_THREADS, 0, s>>>(g, idt, irho, a, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- energy / mass
// z ln z for positive finite z, else 0 (the test on the bit pattern: an FP64 comparison
// would take an FP64-pipe slot)
__device__ __forceinline__ double xlogx(double z) { return pos_bits(z) ? z * table_log<>(z) : 0.0; }
// 0 <= x <= 1 on the bit pattern (-0 included, NaN excluded)
__device__ __forceinline__ bool in_closed_unit(double x) {
    const long long b = __double_as_longlong(x);
    return (unsigned long long)b <= 0x3ff0000000000000ULL || b == (long long)0x8000000000000000ULL;
}

// E~ = sum [e1 + e2 + gamma/2 sum_d ((D+ phi)^2 + (D- phi)^2)/2] dx dy (Eqs. relations,
// freeenergy) and sum u dx dy, as per-block partials [energy | mass].
template <int DIM>
__global__ void __launch_bounds__(256) energy_kernel(Geom g, Coef k, const double* __restrict__ X,
                                                     Red red, int* flags, Members mb) {
    __shared__ double sh[32];
    const int N = g.N;
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    member_coef(mb, m, k);
    X += (size_t)m * mb.vs;
    flags += m;
    red = member_red(red, mb, m);
    const double* __restrict__ U = X;
    const double* __restrict__ V = X + N;
    double e_acc = 0.0, m_acc = 0.0;
    int flag = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int x, y, z;
        decode_cell<DIM>(g, c, x, y, z);
        const double u = U[c], v = V[c];
        const double p = u + v, q = u - v;
        // 1 - p, 1 - q: plain differences, or correctly rounded where a lane of the warp is
        // within 2^-6 of a pure phase (the loop's trip count varies by lane: vote among the
        // lanes still in it)
        double mp = 1.0 - p, mq = 1.0 - q;
        if (__any_sync(__activemask(), near_pure2(2.0 * p) || near_pure2(2.0 * q))) one_minus_pq(u, v, mp, mq);
        if (!(in_closed_unit(p) && in_closed_unit(q))) flag |= 1;
        double e = 0.5 * k.alpha * u * (1.0 - u) - 0.5 * k.beta * v * v
                 + k.theta * (xlogx(p) + xlogx(mp) + xlogx(q) + xlogx(mq));
        // gradient part gamma/2 * 1/2 * sum over D+ and D- of both fields and all axes: a
        // face's difference is the D+ of one cell and the D- of the next (both zero at a
        // Neumann wall, where the neighbour is the cell itself), so the sum over cells of
        // (D+)^2 + (D-)^2 is twice that of (D+)^2 alone
        double gr = 0.0;
#pragma unroll
        for (int f = 1; f < 2 * DIM; f += 2) {
            const int n = face_nb<DIM>(g, x, y, z, f);
            const double du = U[n] - u, dv = V[n] - v;
            gr = fma(fma(du, du, dv * dv), face_ih2(g, f), gr);
        }
        e = fma(0.5 * k.gamma, gr, e);
        e_acc += e;
        m_acc += u;
    }
    if (flag) atomicOr(flags, flag);
    double t = block_sum_red(e_acc, sh);
    if (threadIdx.x == 0) red.partial[blockIdx.x] = t * g.vol;
    t = block_sum_red(m_acc, sh);
    if (threadIdx.x == 0) red.partial[gridDim.x + blockIdx.x] = t * g.vol;
    finish_reduction(red, 2, sh);
}

cudaError_t launch_energy(const Geom& g, const Coef& k, const double* X, Red red, int* flags, cudaStream_t s,
                          const Members& mb) {
    const dim3 nb(red_grid(g.N), mb.count);
    if (g.dim == 3) energy_kernel<3><<<nb, RED_THREADS, 0, s>>>(g, k, X, red, flags, mb);
    else energy_kernel<2><<<nb, RED_THREADS, 0, s>>>(g, k, X, red, flags, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- linearisation
// Per-cell derivative data of F at the accepted iterate X (G = [Gu | Gv | c] from
// pass A at the same X):  cu = dc/du1, cv = dc/dv1 (c at the midpoint, so each picks
// up a factor 1/2), du = -alpha/2 + theta (dphi/dp1 + dpsi/dq1), xc = theta (dphi/dp1 - dpsi/dq1).
// The midpoint sums are formed in double; the derivative arithmetic runs in the
// Jacobian's precision T (double, or float in the mixed form).
template <typename T>
__global__ void __launch_bounds__(256) linearize_kernel(Geom g, Coef k, const double* __restrict__ X,
                                                        const double* __restrict__ X0,
                                                        const double* __restrict__ G, Cache<T> C,
                                                        double ssign) {
    const int N = g.N;
    const T theta = (T)k.theta, halpha = (T)(0.5 * k.alpha);
    const T sgn = (T)ssign;
    // uniform trip count: every lane of a warp takes part in the term-count vote
    const int stride = gridDim.x * blockDim.x;
    const int iters = (N + stride - 1) / stride;
    for (int it = 0; it < iters; ++it) {
        const int c0 = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const bool live = c0 < N;
        const int c = live ? c0 : N - 1;
        const double u1 = X[c], v1 = X[N + c], u0 = X0[c], v0 = X0[N + c];
        // zeta, 1 - zeta and sigma of p and q in double (midpoint_pq2: accurate near the pure
        // phases, where the increments of u and v may cancel), then precision T
        const Midpoint2 m2 = midpoint_pq2_fast(u1, v1, u0, v0);
        const double su = u1 + u0, sv = v1 + v0;
        const T half = (T)0.5;
        const T zp = half * (T)m2.zp, omp = half * (T)m2.omp, zq = half * (T)m2.zq, omq = half * (T)m2.omq;
        const T sp = half * (T)m2.sp, sq = half * (T)m2.sq;
        const T ub = half * (T)su, vb = half * (T)sv;
        const T w = (T)0.25 - vb * vb;
        // ssign = -1: derivative in the start value (phi^S is even in sigma)
        T dp, dq;
        dphi_pair<T>(zp, omp, sgn * sp, zq, omq, sgn * sq, k.S, dp, dq);
        if (!live) continue;
        const T A = theta * dp, B = theta * dq;
        C.c[c] = (T)G[2 * N + c];
        C.cu[c] = (T)0.5 * ((T)1 - (T)2 * ub) * w;
        C.cv[c] = -ub * ((T)1 - ub) * vb;
        C.Gu[c] = (T)G[c];
        C.Gv[c] = (T)G[N + c];
        C.du[c] = -halpha + A + B;
        C.xc[c] = A - B;
    }
}

template <typename T>
cudaError_t launch_linearize(const Geom& g, const Coef& k, const double* X, const double* X0,
                             const double* G, Cache<T> cache, cudaStream_t s, int wrt_x0) {
    cudaError_t e = set_taylor_constants(k.S);
    if (e != cudaSuccess) return e;
    linearize_kernel<T><<<grid_for(g.N, 256), 256, 0, s>>>(g, k, X, X0, G, cache, wrt_x0 ? -1.0 : 1.0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- adjoint
// -mu^T dF/dp for p = alpha, beta, theta, gamma at (X1, X0).  The coefficients enter
// only G~ (linearly), so with A(g) = -div(c~ grad g) (symmetric) and
// q_u = A(mu_u), q_v = c mu_v / rho:
//   -mu^T dF/dp = -sum_cells [dG_u/dp q_u + dG_v/dp q_v],
//   dG/dalpha = (-(u1+u0-1)/2, 0), dG/dbeta = (0, -(v1+v0)/2),
//   dG/dtheta = (phi + psi, phi - psi), dG/dgamma = -(Delta(u1+u0), Delta(v1+v0))/2.
template <int DIM>
__global__ void __launch_bounds__(256) param_grad_kernel(Geom g, Coef k, const double* __restrict__ X1,
                                                         const double* __restrict__ X0,
                                                         const double* __restrict__ G,
                                                         const double* __restrict__ mu, Red red, int* flags) {
    __shared__ double sh[32];
    const int N = g.N;
    const double* __restrict__ cm = G + 2 * N;
    const double irho = 1.0 / k.rho;   // once per thread: this kernel runs once per adjoint step
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int flag = 0;
    const int stride = gridDim.x * blockDim.x;
    const int iters = (N + stride - 1) / stride;
    for (int it = 0; it < iters; ++it) {
        const int c = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
        const bool live = c < N;
        const int cc = live ? c : N - 1;
        int x, y, z;
        decode_cell<DIM>(g, cc, x, y, z);
        const double u1 = X1[cc], v1 = X1[N + cc], u0 = X0[cc], v0 = X0[N + cc];
        const double su = u1 + u0, sv = v1 + v0;
        const double c0 = cm[cc], mu_u = mu[cc];
        double lu = 0.0, lv = 0.0, qu = 0.0;
#pragma unroll
        for (int f = 0; f < 2 * DIM; ++f) {
            const int n = face_nb<DIM>(g, x, y, z, f);
            const double w = face_weight<DIM, double>(g, x, y, z, f);
            lu = fma(X1[n] + X0[n] - su, w, lu);
            lv = fma(X1[N + n] + X0[N + n] - sv, w, lv);
            qu -= w * 0.5 * (c0 + cm[n]) * (mu[n] - mu_u);
        }
        const double qv = c0 * mu[N + cc] * irho;
        const Midpoint2 m2 = midpoint_pq2(u1, v1, u0, v0);
        const bool ok = m2.zp > 0.0 && m2.omp > 0.0 && m2.zq > 0.0 && m2.omq > 0.0;
        if (live && !ok) flag |= 1;
        SeriesArgs ap, aq;
        series_args2(ok ? m2.zp : 1.0, ok ? m2.omp : 1.0, m2.sp, ok ? m2.zq : 1.0, ok ? m2.omq : 1.0, m2.sq, ap,
                     aq);
        const int K = series_terms(max_nonneg(ap.ra, ap.rb, aq.ra, aq.rb), k.S);
        const double phi = phi_series<>(ap, K), psi = phi_series<>(aq, K);
        if (live && ok) {
            acc[0] += 0.5 * (su - 1.0) * qu;
            acc[1] += 0.5 * sv * qv;
            acc[2] -= (phi + psi) * qu + (phi - psi) * qv;
            acc[3] += 0.5 * (lu * qu + lv * qv);
        }
    }
    if (flag) atomicOr(flags, flag);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const double t = block_sum_red(acc[v], sh);
        if (threadIdx.x == 0) red.partial[(size_t)v * gridDim.x + blockIdx.x] = t;
    }
    finish_reduction(red, 4, sh);
}

cudaError_t launch_param_grad(const Geom& g, const Coef& k, const double* X1, const double* X0,
                              const double* G, const double* mu, Red red, int* flags, cudaStream_t s) {
    cudaError_t e = set_taylor_constants(k.S);
    if (e != cudaSuccess) return e;
    if (g.dim == 3) param_grad_kernel<3><<<red_grid(g.N), RED_THREADS, 0, s>>>(g, k, X1, X0, G, mu, red, flags);
    else param_grad_kernel<2><<<red_grid(g.N), RED_THREADS, 0, s>>>(g, k, X1, X0, G, mu, red, flags);
    return cudaGetLastError();
}

// Loss of the final state and its gradient.  E~ as in energy_kernel; its derivative in
// u at a cell is dx dy [alpha/2 (1 - 2u) + theta Phi'(u+v) + theta Phi'(u-v) - gamma Delta u]
// (every face difference enters E~ once as a D+ and once as a D- term), in v
// dx dy [-beta v + theta Phi'(u+v) - theta Phi'(u-v) - gamma Delta v], Phi'(z) = ln z - ln(1-z).
template <int DIM>
__global__ void __launch_bounds__(256) loss_grad_kernel(Geom g, Coef k, const double* __restrict__ X,
                                                        const double* __restrict__ T, double wE, double wM,
                                                        double* __restrict__ lam, Red red, int* flags) {
    __shared__ double sh[32];
    const int N = g.N;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int flag = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        int x, y, z;
        decode_cell<DIM>(g, c, x, y, z);
        const double u = X[c], v = X[N + c];
        const double p = u + v, q = u - v;
        double mp, mq;                                           // 1 - p, 1 - q
        one_minus_pq(u, v, mp, mq);
        if (!(in_unit(p) && in_unit(q))) flag |= 1;
        const double lp = table_log<>(p), lp1 = table_log<>(mp), lq = table_log<>(q), lq1 = table_log<>(mq);
        double lapu = 0.0, lapv = 0.0, gr = 0.0;
#pragma unroll
        for (int f = 0; f < 2 * DIM; ++f) {
            const int n = face_nb<DIM>(g, x, y, z, f);
            const double du = X[n] - u, dv = X[N + n] - v, ih2 = face_ih2(g, f);
            lapu = fma(du, ih2, lapu);
            lapv = fma(dv, ih2, lapv);
            gr = fma(du * du + dv * dv, ih2, gr);
        }
        const double eu = u - T[c], ev = v - T[N + c];
        const double dEu = 0.5 * k.alpha * (1.0 - 2.0 * u) + k.theta * ((lp - lp1) + (lq - lq1)) - k.gamma * lapu;
        const double dEv = -k.beta * v + k.theta * ((lp - lp1) - (lq - lq1)) - k.gamma * lapv;
        lam[c] = g.vol * (wE * dEu + wM * eu);
        lam[N + c] = g.vol * (wE * dEv + wM * ev);
        const double xl = p * lp + mp * lp1 + q * lq + mq * lq1;
        const double e = 0.5 * k.alpha * u * (1.0 - u) - 0.5 * k.beta * v * v + k.theta * xl + 0.25 * k.gamma * gr;
        acc[0] += wE * e + 0.5 * wM * (eu * eu + ev * ev);
        acc[1] += wE * 0.5 * u * (1.0 - u);
        acc[2] -= wE * 0.5 * v * v;
        acc[3] += wE * xl;
        acc[4] += wE * 0.25 * gr;
    }
    if (flag) atomicOr(flags, flag);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        const double t = block_sum_red(acc[v], sh);
        if (threadIdx.x == 0) red.partial[(size_t)v * gridDim.x + blockIdx.x] = t * g.vol;
    }
    finish_reduction(red, 5, sh);
}

cudaError_t launch_loss_grad(const Geom& g, const Coef& k, const double* X, const double* target, double wE,
                             double wM, double* lam, Red red, int* flags, cudaStream_t s) {
    cudaError_t e = set_taylor_constants(k.S);
    if (e != cudaSuccess) return e;
    if (g.dim == 3) loss_grad_kernel<3><<<red_grid(g.N), RED_THREADS, 0, s>>>(g, k, X, target, wE, wM, lam, red, flags);
    else loss_grad_kernel<2><<<red_grid(g.N), RED_THREADS, 0, s>>>(g, k, X, target, wE, wM, lam, red, flags);
    return cudaGetLastError();
}
__global__ void table_log_kernel(const double* __restrict__ x, double* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = table_log<>(x[i]);
}

cudaError_t launch_table_log(const double* x, double* y, long long n, cudaStream_t s) {
    cudaError_t e = set_taylor_constants(1);
    if (e != cudaSuccess) return e;
    table_log_kernel<<<RED_BLOCKS, 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

template cudaError_t launch_linearize<double>(const Geom&, const Coef&, const double*, const double*,
                                              const double*, Cache<double>, cudaStream_t, int);
template cudaError_t launch_linearize<float>(const Geom&, const Coef&, const double*, const double*,
                                             const double*, Cache<float>, cudaStream_t, int);

}  // namespace acac
