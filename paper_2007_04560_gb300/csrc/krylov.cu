// Vector kernels of the restarted GMRES of Sec. 3.1 (Eq. hjacobi): block dot
// products against the Arnoldi basis with warp-shuffle reductions, the classical
// Gram–Schmidt update, norms, scaling, the basis combination V y and the
// precision boundary between the FP64 Newton vectors and the Krylov vectors.
//
// Reductions are two-stage and deterministic: every kernel writes one partial sum
// per block (RED_BLOCKS blocks, grid-stride loops) and its last block to finish adds
// the partials of each quantity in a fixed order (finish_reduction).
#include "acac_internal.cuh"

namespace acac {

// partial sums of (a - b - c) over n  (mass correction of the Newton direction)
__global__ void sum_pair_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                const double* __restrict__ c, long long n, Red red) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc += (a[i] - b[i]) - c[i];
    const double t = block_sum_red(acc, sh);
    if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
    finish_reduction(red, 1, sh);
}

cudaError_t launch_sum_pair(const double* a, const double* b, const double* c, long long n, Red red,
                            cudaStream_t s) {
    sum_pair_kernel<<<red_grid(n), RED_THREADS, 0, s>>>(a, b, c, n, red);
    return cudaGetLastError();
}

__global__ void norm2_double_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                    Red red) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = b ? a[i] - b[i] : a[i];
        acc = fma(x, x, acc);
    }
    const double t = block_sum_red(acc, sh);
    if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
    finish_reduction(red, 1, sh);
}

cudaError_t launch_norm2_double(const double* a, const double* b, long long n, Red red, cudaStream_t s) {
    norm2_double_kernel<<<red_grid(n), RED_THREADS, 0, s>>>(a, b, n, red);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- V^T w
// Vectors are processed in chunks of up to 8, the chunk width a template parameter (a
// predicated FP64 multiply-add still occupies the FP64 pipe, so a fixed 8-wide loop with
// masked lanes cost 8 products per element whatever the count).  Each thread
// accumulates its share in the Krylov precision; the block and global stages add in
// double, the block stage with one barrier per chunk.
template <typename T, int C>
__device__ __forceinline__ void dot_chunk(const T* __restrict__ V, long long ld, const T* __restrict__ w,
                                          long long n, double* __restrict__ partial, double (*sw)[RED_THREADS / 32]) {
    T acc[C];
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const T wi = w[i];
#pragma unroll
        for (int q = 0; q < C; ++q) acc[q] += V[(size_t)q * ld + i] * wi;
    }
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
        partial[(size_t)threadIdx.x * RED_BLOCKS + blockIdx.x] = t;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) multi_dot_kernel(const T* __restrict__ V, long long ld, int nv,
                                                                const T* __restrict__ w, long long n,
                                                                Red red) {
    __shared__ double sw[8][RED_THREADS / 32];
    for (int k0 = 0; k0 < nv; k0 += 8) {
        const T* Vk = V + (size_t)k0 * ld;
        double* pk = red.partial + (size_t)k0 * RED_BLOCKS;
        switch (nv - k0 < 8 ? nv - k0 : 8) {
            case 1: dot_chunk<T, 1>(Vk, ld, w, n, pk, sw); break;
            case 2: dot_chunk<T, 2>(Vk, ld, w, n, pk, sw); break;
            case 3: dot_chunk<T, 3>(Vk, ld, w, n, pk, sw); break;
            case 4: dot_chunk<T, 4>(Vk, ld, w, n, pk, sw); break;
            case 5: dot_chunk<T, 5>(Vk, ld, w, n, pk, sw); break;
            case 6: dot_chunk<T, 6>(Vk, ld, w, n, pk, sw); break;
            case 7: dot_chunk<T, 7>(Vk, ld, w, n, pk, sw); break;
            default: dot_chunk<T, 8>(Vk, ld, w, n, pk, sw); break;
        }
    }
    finish_reduction(red, nv, nullptr);
}

template <typename T>
cudaError_t launch_multi_dot(const T* V, long long ld, int nv, const T* w, long long n, Red red,
                             cudaStream_t s) {
    multi_dot_kernel<T><<<red_grid(n), RED_THREADS, 0, s>>>(V, ld, nv, w, n, red);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- w -= V h  (+ ||w||^2)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) cgs_update_kernel(const T* __restrict__ V, long long ld, int nv,
                                                                 const double* __restrict__ h, T* __restrict__ w,
                                                                 long long n, int want_norm, Red red) {
    __shared__ double sh[32];
    __shared__ T hs[MAX_RESTART + 1];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) hs[k] = (T)h[k];
    __syncthreads();
    T acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T s = 0;
        int k = 0;
        for (; k + 4 <= nv; k += 4)
            s += hs[k] * V[(size_t)k * ld + i] + hs[k + 1] * V[(size_t)(k + 1) * ld + i]
               + hs[k + 2] * V[(size_t)(k + 2) * ld + i] + hs[k + 3] * V[(size_t)(k + 3) * ld + i];
        for (; k < nv; ++k) s += hs[k] * V[(size_t)k * ld + i];
        const T wn = w[i] - s;
        w[i] = wn;
        acc += wn * wn;
    }
    if (want_norm) {
        const double t = block_sum_red((double)acc, sh);
        if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
        finish_reduction(red, 1, sh);
    }
}

template <typename T>
cudaError_t launch_cgs_update(const T* V, long long ld, int nv, const double* h, T* w, long long n,
                              int want_norm, Red red, cudaStream_t s) {
    cgs_update_kernel<T><<<red_grid(n), RED_THREADS, 0, s>>>(V, ld, nv, h, w, n, want_norm, red);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- out = w / alpha (alpha on device)
template <typename T>
__global__ void scale_from_kernel(const T* __restrict__ w, const double* __restrict__ alpha,
                                  T* __restrict__ out, long long n) {
    // alpha holds ||w||^2; one thread per block forms 1/||w|| (an FP64 square root
    // and division per thread would cost more than the scaling itself)
    __shared__ T s_inv;
    if (threadIdx.x == 0) s_inv = (T)(1.0 / sqrt(alpha[0]));
    __syncthreads();
    const T inv = s_inv;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = w[i] * inv;
}

template <typename T>
cudaError_t launch_scale_from(const T* w, const double* alpha_dev, T* out, long long n,
                              cudaStream_t s) {
    scale_from_kernel<T><<<red_grid(n), RED_THREADS, 0, s>>>(w, alpha_dev, out, n);
    return cudaGetLastError();
}

template <typename T>
__global__ void to_krylov_kernel(const double* __restrict__ x, double scale, T* __restrict__ out,
                                 long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)(x[i] * scale);
}

template <typename T>
cudaError_t launch_to_krylov(const double* x, double scale, T* out, long long n, cudaStream_t s) {
    to_krylov_kernel<T><<<red_grid(n), RED_THREADS, 0, s>>>(x, scale, out, n);
    return cudaGetLastError();
}

// out = sum_k y_k V_k
template <typename T>
__global__ void lincomb_kernel(const T* __restrict__ V, long long ld, int nv, const double* __restrict__ y,
                               T* __restrict__ out, long long n) {
    __shared__ T ys[MAX_RESTART + 1];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) ys[k] = (T)y[k];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T s = 0;
        for (int k = 0; k < nv; ++k) s += ys[k] * V[(size_t)k * ld + i];
        out[i] = s;
    }
}

template <typename T>
cudaError_t launch_lincomb(const T* V, long long ld, int nv, const double* y, T* out, long long n,
                           cudaStream_t s) {
    lincomb_kernel<T><<<red_grid(n), RED_THREADS, 0, s>>>(V, ld, nv, y, out, n);
    return cudaGetLastError();
}

template <typename T>
__global__ void axpy_to_double_kernel(double a, const T* __restrict__ x, double* __restrict__ y,
                                      long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = fma(a, (double)x[i], y[i]);
}

template <typename T>
cudaError_t launch_axpy_to_double(double a, const T* x, double* y, long long n, cudaStream_t s) {
    axpy_to_double_kernel<T><<<red_grid(n), RED_THREADS, 0, s>>>(a, x, y, n);
    return cudaGetLastError();
}

// r = b - Ax (double), partial sums of ||r||^2
template <typename T>
__global__ void residual_restart_kernel(const double* __restrict__ b, const T* __restrict__ Ax,
                                        double* __restrict__ r, long long n, Red red) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double ri = b[i] - (double)Ax[i];
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    const double t = block_sum_red(acc, sh);
    if (threadIdx.x == 0) red.partial[blockIdx.x] = t;
    finish_reduction(red, 1, sh);
}

template <typename T>
cudaError_t launch_residual_restart(const double* b, const T* Ax, double* r, long long n, Red red,
                                    cudaStream_t s) {
    residual_restart_kernel<T><<<red_grid(n), RED_THREADS, 0, s>>>(b, Ax, r, n, red);
    return cudaGetLastError();
}

#define INST(T)                                                                                     \
    template cudaError_t launch_multi_dot<T>(const T*, long long, int, const T*, long long, Red,    \
                                             cudaStream_t);                                         \
    template cudaError_t launch_cgs_update<T>(const T*, long long, int, const double*, T*, long long, \
                                              int, Red, cudaStream_t);                              \
    template cudaError_t launch_scale_from<T>(const T*, const double*, T*, long long, cudaStream_t); \
    template cudaError_t launch_to_krylov<T>(const double*, double, T*, long long, cudaStream_t);   \
    template cudaError_t launch_lincomb<T>(const T*, long long, int, const double*, T*, long long,  \
                                           cudaStream_t);                                           \
    template cudaError_t launch_axpy_to_double<T>(double, const T*, double*, long long, cudaStream_t); \
    template cudaError_t launch_residual_restart<T>(const double*, const T*, double*, long long,    \
                                                    Red, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace acac
