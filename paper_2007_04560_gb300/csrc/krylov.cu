// Vector kernels of the restarted GMRES of Sec. 3.1 (Eq. hjacobi): block dot
// products against the Arnoldi basis with warp-shuffle reductions, the classical
// Gram–Schmidt update, norms, scaling, the basis combination V y, the precision
// boundary between the FP64 Newton vectors and the Krylov vectors, and the small
// per-member GMRES steps (Givens rotations, convergence test, back substitution).
//
// Reductions are two-stage and deterministic: every kernel writes one partial sum
// per block (at most RED_BLOCKS blocks per member, grid-stride loops) and the member's
// last block to finish adds the partials of each quantity in a fixed order
// (finish_reduction).  Member m of an ensemble is blockIdx.y; its vectors sit at
// m * mb.vs, its device scalars at m * mb.rs.
#include <stdint.h>
#include <string.h>

#include "acac_internal.cuh"

namespace acac {

static dim3 vgrid(long long n, const Members& mb) { return dim3(red_grid(n), mb.count); }

// Element packs.  A thread takes P = 4 consecutive elements per step, loaded with 16-byte
// vector loads when every pointer of the launch is 16-byte aligned (the handle's buffers
// and member strides are), so that more bytes are in flight per thread; otherwise (P = 1)
// element by element.  Elements past the last whole pack are taken one by one.
template <typename T, int P>
struct Pk {
    T v[P];
};
template <typename T, int P>
__device__ __forceinline__ Pk<T, P> ldp(const T* __restrict__ p, long long i) {
    Pk<T, P> r;
    if constexpr (P * sizeof(T) % 16 == 0) {
        const uint4* q = reinterpret_cast<const uint4*>(p + i * P);
#pragma unroll
        for (int k = 0; k < (int)(P * sizeof(T) / 16); ++k) {
            const uint4 u = q[k];
            memcpy(&r.v[k * (16 / sizeof(T))], &u, 16);
        }
    } else {
#pragma unroll
        for (int k = 0; k < P; ++k) r.v[k] = p[i * P + k];
    }
    return r;
}
template <typename T, int P>
__device__ __forceinline__ void stp(T* __restrict__ p, long long i, const Pk<T, P>& r) {
    if constexpr (P * sizeof(T) % 16 == 0) {
        uint4* q = reinterpret_cast<uint4*>(p + i * P);
#pragma unroll
        for (int k = 0; k < (int)(P * sizeof(T) / 16); ++k) {
            uint4 u;
            memcpy(&u, &r.v[k * (16 / sizeof(T))], 16);
            q[k] = u;
        }
    } else {
#pragma unroll
        for (int k = 0; k < P; ++k) p[i * P + k] = r.v[k];
    }
}
// Runs f(pack index) over the whole packs and g(element index) over the remaining elements,
// grid-stride within the member's blocks; with U = 2 two packs per trip, so that the loads
// of both are issued before either is used (twice the bytes in flight per thread).
template <int P, int U = 2, typename F, typename G>
__device__ __forceinline__ void over_packs(long long n, F f, G g) {
    const long long np = n / P;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
    long long i = t0;
    if (U == 2)
        for (; i + st < np; i += 2 * st) {
            f(i);
            f(i + st);
        }
    for (; i < np; i += st) f(i);
    for (long long e = np * P + t0; e < n; e += st) g(e);
}
static bool al16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// partial sums of (a - b - c) over n  (mass correction of the Newton direction)
template <int P>
__global__ void sum_pair_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                const double* __restrict__ c, long long n, Red red, Members mb) {
    __shared__ double sh[32];
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    const size_t o = (size_t)m * mb.vs;
    a += o; b += o; c += o;
    red = member_red(red, mb, m);
    double acc = 0.0;
    over_packs<P>(n, [&](long long i) {
        const Pk<double, P> x = ldp<double, P>(a, i), y = ldp<double, P>(b, i), z = ldp<double, P>(c, i);
#pragma unroll
        for (int k = 0; k < P; ++k) acc += (x.v[k] - y.v[k]) - z.v[k];
    }, [&](long long i) { acc += (a[i] - b[i]) - c[i]; });
    const double t = block_sum_red(acc, sh);
    if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
    finish_reduction(red, 1, sh);
}

cudaError_t launch_sum_pair(const double* a, const double* b, const double* c, long long n, Red red,
                            cudaStream_t s, const Members& mb) {
    if (al16(a) && al16(b) && al16(c)) sum_pair_kernel<4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(a, b, c, n, red, mb);
    else sum_pair_kernel<1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(a, b, c, n, red, mb);
    return cudaGetLastError();
}

template <int P>
__global__ void norm2_double_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                    Red red, Members mb) {
    __shared__ double sh[32];
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    const size_t o = (size_t)m * mb.vs;
    a += o;
    if (b) b += o;
    red = member_red(red, mb, m);
    double acc = 0.0;
    over_packs<P>(n, [&](long long i) {
        const Pk<double, P> x = ldp<double, P>(a, i);
        if (b) {
            const Pk<double, P> y = ldp<double, P>(b, i);
#pragma unroll
            for (int k = 0; k < P; ++k) acc = fma(x.v[k] - y.v[k], x.v[k] - y.v[k], acc);
        } else {
#pragma unroll
            for (int k = 0; k < P; ++k) acc = fma(x.v[k], x.v[k], acc);
        }
    }, [&](long long i) {
        const double x = b ? a[i] - b[i] : a[i];
        acc = fma(x, x, acc);
    });
    const double t = block_sum_red(acc, sh);
    if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
    finish_reduction(red, 1, sh);
}

cudaError_t launch_norm2_double(const double* a, const double* b, long long n, Red red, cudaStream_t s,
                                const Members& mb) {
    if (al16(a) && (!b || al16(b))) norm2_double_kernel<4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(a, b, n, red, mb);
    else norm2_double_kernel<1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(a, b, n, red, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- V^T w
// Vectors are processed in chunks of up to 4, the chunk width a template parameter (a
// predicated multiply-add still occupies its pipe, so a fixed-width loop with masked
// lanes would cost the full width per element whatever the count).  Each thread
// accumulates its share in the Krylov precision; the block and global stages add in
// double, the block stage with one barrier per chunk.
template <typename T, int C, int P>
__device__ __forceinline__ void dot_chunk(const T* __restrict__ V, long long ld, const T* __restrict__ w,
                                          long long n, double* __restrict__ partial, double (*sw)[RED_THREADS / 32]) {
    T acc[C];
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = 0;
    over_packs<P, (C <= 2 ? 2 : 1)>(n, [&](long long i) {
        const Pk<T, P> wi = ldp<T, P>(w, i);
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const Pk<T, P> vq = ldp<T, P>(V + (size_t)q * ld, i);
#pragma unroll
            for (int k = 0; k < P; ++k) acc[q] += vq.v[k] * wi.v[k];
        }
    }, [&](long long i) {
        const T wi = w[i];
#pragma unroll
        for (int q = 0; q < C; ++q) acc[q] += V[(size_t)q * ld + i] * wi;
    });
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < C; ++q) {
        const double t = warp_sum((double)acc[q]);
        if (lane == 0) sw[q][warp] = t;
    }
    __syncthreads();
    if ((int)threadIdx.x < C) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < RED_THREADS / 32; ++k) t += sw[threadIdx.x][k];
        partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
}

// One launch per chunk of up to four vectors, the width a template parameter: the kernel
// keeps only that chunk's packs in registers (it is bound by the bytes in flight, i.e. by
// the resident warps), and chunks of one or two vectors take two packs per trip.
template <typename T, int P, int C>
__global__ void __launch_bounds__(RED_THREADS) multi_dot_kernel(const T* __restrict__ V, long long ld,
                                                                const T* __restrict__ w, long long n,
                                                                Red red, Members mb) {
    __shared__ double sw[8][RED_THREADS / 32];
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    V += (size_t)m * mb.vs;
    w += (size_t)m * mb.vs;
    red = member_red(red, mb, m);
    dot_chunk<T, C, P>(V, ld, w, n, red.partial, sw);
    finish_reduction(red, C, nullptr);
}

template <typename T, int P>
static void multi_dot_chunk(const T* V, long long ld, int c, const T* w, long long n, Red red, cudaStream_t s,
                            const Members& mb) {
    const dim3 g = vgrid(n, mb);
    switch (c) {
        case 1: multi_dot_kernel<T, P, 1><<<g, RED_THREADS, 0, s>>>(V, ld, w, n, red, mb); break;
        case 2: multi_dot_kernel<T, P, 2><<<g, RED_THREADS, 0, s>>>(V, ld, w, n, red, mb); break;
        case 3: multi_dot_kernel<T, P, 3><<<g, RED_THREADS, 0, s>>>(V, ld, w, n, red, mb); break;
        default: multi_dot_kernel<T, P, 4><<<g, RED_THREADS, 0, s>>>(V, ld, w, n, red, mb); break;
    }
}

// h[k] = V_k . w for k < nv: the chunks' results land at red.out + k0 (the launches run in
// stream order and share the partials and the counter)
template <typename T>
cudaError_t launch_multi_dot(const T* V, long long ld, int nv, const T* w, long long n, Red red,
                             cudaStream_t s, const Members& mb) {
    const bool vec = al16(V) && al16(w) && (ld * sizeof(T)) % 16 == 0;
    for (int k0 = 0; k0 < nv; k0 += 4) {
        Red r = red;
        r.out += k0;
        const int c = nv - k0 < 4 ? nv - k0 : 4;
        if (vec) multi_dot_chunk<T, 16 / sizeof(T)>(V + (size_t)k0 * ld, ld, c, w, n, r, s, mb);
        else multi_dot_chunk<T, 1>(V + (size_t)k0 * ld, ld, c, w, n, r, s, mb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- w -= V h  (+ ||w||^2)
template <typename T, int P>
__global__ void __launch_bounds__(RED_THREADS) cgs_update_kernel(const T* __restrict__ V, long long ld, int nv,
                                                                 const double* __restrict__ h, T* __restrict__ w,
                                                                 long long n, int want_norm, Red red, Members mb) {
    __shared__ double sh[32];
    __shared__ T hs[MAX_RESTART + 1];
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    V += (size_t)m * mb.vs;
    w += (size_t)m * mb.vs;
    h += (size_t)m * mb.rs;
    red = member_red(red, mb, m);
    for (int k = threadIdx.x; k < nv; k += blockDim.x) hs[k] = (T)h[k];
    __syncthreads();
    T acc = 0;
    over_packs<P>(n, [&](long long i) {
        Pk<T, P> s;
#pragma unroll
        for (int e = 0; e < P; ++e) s.v[e] = 0;
        for (int k = 0; k < nv; ++k) {
            const Pk<T, P> vk = ldp<T, P>(V + (size_t)k * ld, i);
            const T hk = hs[k];
#pragma unroll
            for (int e = 0; e < P; ++e) s.v[e] += hk * vk.v[e];
        }
        Pk<T, P> wi = ldp<T, P>(w, i);
#pragma unroll
        for (int e = 0; e < P; ++e) {
            wi.v[e] -= s.v[e];
            acc += wi.v[e] * wi.v[e];
        }
        stp<T, P>(w, i, wi);
    }, [&](long long i) {
        T s = 0;
        for (int k = 0; k < nv; ++k) s += hs[k] * V[(size_t)k * ld + i];
        const T wn = w[i] - s;
        w[i] = wn;
        acc += wn * wn;
    });
    if (want_norm) {
        const double t = block_sum_red((double)acc, sh);
        if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
        finish_reduction(red, 1, sh);
    }
}

template <typename T>
cudaError_t launch_cgs_update(const T* V, long long ld, int nv, const double* h, T* w, long long n,
                              int want_norm, Red red, cudaStream_t s, const Members& mb) {
    if (al16(V) && al16(w) && (ld * sizeof(T)) % 16 == 0)
        cgs_update_kernel<T, 4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(V, ld, nv, h, w, n, want_norm, red, mb);
    else
        cgs_update_kernel<T, 1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(V, ld, nv, h, w, n, want_norm, red, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- out = w / alpha (alpha on device)
template <typename T, int P>
__global__ void scale_from_kernel(const T* __restrict__ w, const double* __restrict__ alpha,
                                  T* __restrict__ out, long long n, Members mb) {
    // alpha holds ||w||^2; one thread per block forms 1/||w|| (an FP64 square root
    // and division per thread would cost more than the scaling itself)
    __shared__ T s_inv;
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    w += (size_t)m * mb.vs;
    out += (size_t)m * mb.vs;
    if (threadIdx.x == 0) s_inv = (T)(1.0 / sqrt(alpha[(size_t)m * mb.rs]));
    __syncthreads();
    const T inv = s_inv;
    over_packs<P>(n, [&](long long i) {
        Pk<T, P> x = ldp<T, P>(w, i);
#pragma unroll
        for (int e = 0; e < P; ++e) x.v[e] *= inv;
        stp<T, P>(out, i, x);
    }, [&](long long i) { out[i] = w[i] * inv; });
}

template <typename T>
cudaError_t launch_scale_from(const T* w, const double* alpha_dev, T* out, long long n,
                              cudaStream_t s, const Members& mb) {
    if (al16(w) && al16(out)) scale_from_kernel<T, 4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(w, alpha_dev, out, n, mb);
    else scale_from_kernel<T, 1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(w, alpha_dev, out, n, mb);
    return cudaGetLastError();
}

template <typename T, int P>
__global__ void to_krylov_kernel(const double* __restrict__ x, double scale, T* __restrict__ out,
                                 long long n, Members mb, const double* __restrict__ scale_dev, int sstride) {
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    x += (size_t)m * mb.vs;
    out += (size_t)m * mb.vs;
    // scale / beta with 1/beta correctly rounded, as the host forms it for a single problem
    // (scale is +-1 there: an exact sign)
    if (scale_dev) scale *= 1.0 / scale_dev[(size_t)m * sstride];
    over_packs<P>(n, [&](long long i) {
        const Pk<double, P> a = ldp<double, P>(x, i);
        Pk<T, P> r;
#pragma unroll
        for (int e = 0; e < P; ++e) r.v[e] = from_dbl<T>(a.v[e] * scale);
        stp<T, P>(out, i, r);
    }, [&](long long i) { out[i] = from_dbl<T>(x[i] * scale); });
}

template <typename T>
cudaError_t launch_to_krylov(const double* x, double scale, T* out, long long n, cudaStream_t s,
                             const Members& mb, const double* scale_dev, int sstride) {
    if (al16(x) && al16(out))
        to_krylov_kernel<T, 4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(x, scale, out, n, mb, scale_dev, sstride);
    else
        to_krylov_kernel<T, 1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(x, scale, out, n, mb, scale_dev, sstride);
    return cudaGetLastError();
}

// out = sum_k y_k V_k
template <typename T, int P>
__global__ void lincomb_kernel(const T* __restrict__ V, long long ld, int nv, const double* __restrict__ y,
                               T* __restrict__ out, long long n, Members mb, const int* __restrict__ nv_dev) {
    __shared__ T ys[MAX_RESTART + 1];
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    if (nv_dev) nv = nv_dev[m];
    V += (size_t)m * mb.vs;
    out += (size_t)m * mb.vs;
    y += (size_t)m * mb.rs;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) ys[k] = (T)y[k];
    __syncthreads();
    over_packs<P>(n, [&](long long i) {
        Pk<T, P> s;
#pragma unroll
        for (int e = 0; e < P; ++e) s.v[e] = 0;
        for (int k = 0; k < nv; ++k) {
            const Pk<T, P> vk = ldp<T, P>(V + (size_t)k * ld, i);
#pragma unroll
            for (int e = 0; e < P; ++e) s.v[e] += ys[k] * vk.v[e];
        }
        stp<T, P>(out, i, s);
    }, [&](long long i) {
        T s = 0;
        for (int k = 0; k < nv; ++k) s += ys[k] * V[(size_t)k * ld + i];
        out[i] = s;
    });
}

template <typename T>
cudaError_t launch_lincomb(const T* V, long long ld, int nv, const double* y, T* out, long long n,
                           cudaStream_t s, const Members& mb, const int* nv_dev) {
    if (al16(V) && al16(out) && (ld * sizeof(T)) % 16 == 0)
        lincomb_kernel<T, 4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(V, ld, nv, y, out, n, mb, nv_dev);
    else
        lincomb_kernel<T, 1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(V, ld, nv, y, out, n, mb, nv_dev);
    return cudaGetLastError();
}

template <typename T, int P>
__global__ void axpy_to_double_kernel(double a, const T* __restrict__ x, double* __restrict__ y,
                                      long long n, Members mb) {
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    x += (size_t)m * mb.vs;
    y += (size_t)m * mb.vs;
    over_packs<P>(n, [&](long long i) {
        const Pk<T, P> xi = ldp<T, P>(x, i);
        Pk<double, P> yi = ldp<double, P>(y, i);
#pragma unroll
        for (int e = 0; e < P; ++e) yi.v[e] = fma(a, to_dbl<T>(xi.v[e]), yi.v[e]);
        stp<double, P>(y, i, yi);
    }, [&](long long i) { y[i] = fma(a, to_dbl<T>(x[i]), y[i]); });
}

template <typename T>
cudaError_t launch_axpy_to_double(double a, const T* x, double* y, long long n, cudaStream_t s,
                                  const Members& mb) {
    if (al16(x) && al16(y)) axpy_to_double_kernel<T, 4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(a, x, y, n, mb);
    else axpy_to_double_kernel<T, 1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(a, x, y, n, mb);
    return cudaGetLastError();
}

// r = bsign b - Ax (double; bsign = +-1, an exact sign), partial sums of ||r||^2
template <typename T, int P>
__global__ void residual_restart_kernel(const double* __restrict__ b, double bsign, const T* __restrict__ Ax,
                                        double* __restrict__ r, long long n, Red red, Members mb) {
    __shared__ double sh[32];
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    b += (size_t)m * mb.vs;
    Ax += (size_t)m * mb.vs;
    r += (size_t)m * mb.vs;
    red = member_red(red, mb, m);
    double acc = 0.0;
    over_packs<P>(n, [&](long long i) {
        const Pk<double, P> bi = ldp<double, P>(b, i);
        const Pk<T, P> ai = ldp<T, P>(Ax, i);
        Pk<double, P> ri;
#pragma unroll
        for (int e = 0; e < P; ++e) {
            ri.v[e] = bsign * bi.v[e] - to_dbl<T>(ai.v[e]);
            acc = fma(ri.v[e], ri.v[e], acc);
        }
        stp<double, P>(r, i, ri);
    }, [&](long long i) {
        const double ri = bsign * b[i] - to_dbl<T>(Ax[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    });
    const double t = block_sum_red(acc, sh);
    if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
    finish_reduction(red, 1, sh);
}

template <typename T>
cudaError_t launch_residual_restart(const double* b, double bsign, const T* Ax, double* r, long long n, Red red,
                                    cudaStream_t s, const Members& mb) {
    if (al16(b) && al16(Ax) && al16(r))
        residual_restart_kernel<T, 4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(b, bsign, Ax, r, n, red, mb);
    else
        residual_restart_kernel<T, 1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(b, bsign, Ax, r, n, red, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- member copies
template <int P>
__global__ void copy_members_kernel(const double* __restrict__ x, double* __restrict__ y, long long n, Members mb) {
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    x += (size_t)m * mb.vs;
    y += (size_t)m * mb.vs;
    over_packs<P>(n, [&](long long i) { stp<double, P>(y, i, ldp<double, P>(x, i)); }, [&](long long i) { y[i] = x[i]; });
}

cudaError_t launch_copy_members(const double* x, double* y, long long n, cudaStream_t s, const Members& mb) {
    if (al16(x) && al16(y)) copy_members_kernel<4><<<vgrid(n, mb), RED_THREADS, 0, s>>>(x, y, n, mb);
    else copy_members_kernel<1><<<vgrid(n, mb), RED_THREADS, 0, s>>>(x, y, n, mb);
    return cudaGetLastError();
}

// u, v: the ensemble's fields (member m at m * N); X: member states [u | v] at m * vs
template <int P>
__global__ void pack_members_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                    double* __restrict__ X, long long N, int to_state, Members mb) {
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    double* Xm = X + (size_t)m * mb.vs;
    double* um = const_cast<double*>(u) + (size_t)m * N;
    double* vm = const_cast<double*>(v) + (size_t)m * N;
    if (to_state)
        over_packs<P>(N, [&](long long i) {
            stp<double, P>(Xm, i, ldp<double, P>(um, i));
            stp<double, P>(Xm + N, i, ldp<double, P>(vm, i));
        }, [&](long long i) {
            Xm[i] = um[i];
            Xm[N + i] = vm[i];
        });
    else
        over_packs<P>(N, [&](long long i) {
            stp<double, P>(um, i, ldp<double, P>(Xm, i));
            stp<double, P>(vm, i, ldp<double, P>(Xm + N, i));
        }, [&](long long i) {
            um[i] = Xm[i];
            vm[i] = Xm[N + i];
        });
}

cudaError_t launch_pack_members(const double* u, const double* v, double* X, long long N, int to_state,
                                cudaStream_t s, const Members& mb) {
    if (al16(u) && al16(v) && al16(X) && N % 2 == 0 && mb.vs % 2 == 0)
        pack_members_kernel<4><<<vgrid(N, mb), RED_THREADS, 0, s>>>(u, v, X, N, to_state, mb);
    else
        pack_members_kernel<1><<<vgrid(N, mb), RED_THREADS, 0, s>>>(u, v, X, N, to_state, mb);
    return cudaGetLastError();
}

// X = [u | v] per member and, when Xp is set, partial sums of ||X - Xp||^2 (the step
// predictor's change of state, Sec. 3.2): one pass over the new state instead of a copy
// followed by a norm.  P = 4 needs every pointer 16-byte aligned and N even (member and
// field offsets of N doubles).
template <int P>
__global__ void pack_state_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                  double* __restrict__ X, const double* __restrict__ Xp, long long N, Red red,
                                  Members mb) {
    __shared__ double sh[32];
    const int m = blockIdx.y;
    if (member_off(mb, m)) return;
    u += (size_t)m * N;
    v += (size_t)m * N;
    X += (size_t)m * mb.vs;
    if (Xp) Xp += (size_t)m * mb.vs;
    double acc = 0.0;
    over_packs<P>(N, [&](long long i) {
        const Pk<double, P> a = ldp<double, P>(u, i), b = ldp<double, P>(v, i);
        stp<double, P>(X, i, a);
        stp<double, P>(X + N, i, b);
        if (Xp) {
            const Pk<double, P> pa = ldp<double, P>(Xp, i), pb = ldp<double, P>(Xp + N, i);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                acc = fma(a.v[k] - pa.v[k], a.v[k] - pa.v[k], acc);
                acc = fma(b.v[k] - pb.v[k], b.v[k] - pb.v[k], acc);
            }
        }
    }, [&](long long i) {
        const double a = u[i], b = v[i];
        X[i] = a;
        X[N + i] = b;
        if (Xp) {
            acc = fma(a - Xp[i], a - Xp[i], acc);
            acc = fma(b - Xp[N + i], b - Xp[N + i], acc);
        }
    });
    if (!Xp) return;   // uniform over the grid
    red = member_red(red, mb, m);
    const double t = block_sum_red(acc, sh);
    if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
    finish_reduction(red, 1, sh);
}

cudaError_t launch_pack_state(const double* u, const double* v, double* X, const double* Xp, long long N, Red red,
                              cudaStream_t s, const Members& mb) {
    if (al16(u) && al16(v) && al16(X) && (!Xp || al16(Xp)) && N % 2 == 0 && mb.vs % 2 == 0)
        pack_state_kernel<4><<<vgrid(N, mb), RED_THREADS, 0, s>>>(u, v, X, Xp, N, red, mb);
    else
        pack_state_kernel<1><<<vgrid(N, mb), RED_THREADS, 0, s>>>(u, v, X, Xp, N, red, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- GMRES steps per member
// One thread per member: the steps are O(j) scalar operations, negligible beside the
// vector kernels of the Arnoldi step, and run on the device so that the host launches a
// whole restart cycle without reading anything back in between.
__global__ void gmres_start_kernel(GmresHead* __restrict__ head, GmresWork* __restrict__ work,
                                   const int* __restrict__ on, int* __restrict__ gon, int count) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count) return;
    const int o = on ? on[m] : 1;
    gon[m] = o;
    if (o) work[m].g[0] = head[m].beta;
}

cudaError_t launch_gmres_start(GmresHead* head, GmresWork* work, const int* on, int* gon, int count,
                               cudaStream_t s) {
    gmres_start_kernel<<<(count + 127) / 128, 128, 0, s>>>(head, work, on, gon, count);
    return cudaGetLastError();
}

// Column j of the Hessenberg matrix: rotated by the previous rotations, then the new
// rotation zeroes its subdiagonal entry; the rotated right-hand side g gives the residual
// norm |g_{j+1}| of the minimiser over the j + 1 directions.
__global__ void gmres_givens_kernel(GmresHead* __restrict__ head, GmresWork* __restrict__ work,
                                    const double* __restrict__ red, int rs, int j, int passes,
                                    int* __restrict__ gon, int count) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count || !gon[m]) return;
    const double* r = red + (size_t)m * rs;
    GmresWork& W = work[m];
    GmresHead& H = head[m];
    double* R = W.R + (size_t)j * MAX_RESTART;
    for (int i = 0; i <= j; ++i) R[i] = passes == 2 ? r[i] + r[(MAX_RESTART + 1) + i] : r[i];
    const double hn = sqrt(r[2 * (MAX_RESTART + 1)]);
    for (int i = 0; i < j; ++i) {
        const double a = R[i], b = R[i + 1];
        R[i] = W.cs[i] * a + W.sn[i] * b;
        R[i + 1] = -W.sn[i] * a + W.cs[i] * b;
    }
    const double rho = hypot(R[j], hn);
    W.cs[j] = R[j] / rho;
    W.sn[j] = hn / rho;
    R[j] = rho;
    W.g[j + 1] = -W.sn[j] * W.g[j];
    W.g[j] = W.cs[j] * W.g[j];
    const double resid = fabs(W.g[j + 1]);
    H.resid = resid;
    H.its += 1;
    H.k = j + 1;
    if (!(resid == resid) || !isfinite(rho)) {
        H.status = GMRES_NONFINITE;
        gon[m] = 0;
    } else if (resid <= H.tol || H.its >= H.maxit || hn == 0.0) {
        H.status = (resid <= H.tol || hn == 0.0) ? GMRES_CONVERGED : GMRES_LIMIT;
        gon[m] = 0;
    }
}

cudaError_t launch_gmres_givens(GmresHead* head, GmresWork* work, const double* red, int rs, int j, int passes,
                                int* gon, int count, cudaStream_t s) {
    gmres_givens_kernel<<<(count + 127) / 128, 128, 0, s>>>(head, work, red, rs, j, passes, gon, count);
    return cudaGetLastError();
}

// y = R(0:k, 0:k)^-1 g(0:k) by back substitution
__global__ void gmres_solve_kernel(const GmresHead* __restrict__ head, const GmresWork* __restrict__ work,
                                   const int* __restrict__ on, double* __restrict__ y, int rs,
                                   int* __restrict__ kcnt, int count) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= count || (on && !on[m])) return;
    const int k = head[m].k;
    const GmresWork& W = work[m];
    double* yv = y + (size_t)m * rs;
    kcnt[m] = k;
    for (int i = k - 1; i >= 0; --i) {
        double s = W.g[i];
        for (int jj = i + 1; jj < k; ++jj) s -= W.R[(size_t)jj * MAX_RESTART + i] * yv[jj];
        yv[i] = s / W.R[(size_t)i * MAX_RESTART + i];
    }
}

cudaError_t launch_gmres_solve(const GmresHead* head, const GmresWork* work, const int* on, double* y, int rs,
                               int* kcnt, int count, cudaStream_t s) {
    gmres_solve_kernel<<<(count + 127) / 128, 128, 0, s>>>(head, work, on, y, rs, kcnt, count);
    return cudaGetLastError();
}

#define INST(T)                                                                                     \
    template cudaError_t launch_multi_dot<T>(const T*, long long, int, const T*, long long, Red,    \
                                             cudaStream_t, const Members&);                         \
    template cudaError_t launch_cgs_update<T>(const T*, long long, int, const double*, T*, long long, \
                                              int, Red, cudaStream_t, const Members&);              \
    template cudaError_t launch_scale_from<T>(const T*, const double*, T*, long long, cudaStream_t, \
                                              const Members&);                                      \
    template cudaError_t launch_to_krylov<T>(const double*, double, T*, long long, cudaStream_t,    \
                                             const Members&, const double*, int);                   \
    template cudaError_t launch_lincomb<T>(const T*, long long, int, const double*, T*, long long,  \
                                           cudaStream_t, const Members&, const int*);               \
    template cudaError_t launch_axpy_to_double<T>(double, const T*, double*, long long, cudaStream_t, \
                                                  const Members&);                                  \
    template cudaError_t launch_residual_restart<T>(const double*, double, const T*, double*, long long, \
                                                    Red, cudaStream_t, const Members&);
INST(double)
INST(float)
#undef INST

}  // namespace acac
