// Restricted additive Schwarz preconditioner with ILU(0) subdomain solves
// (Sec. 3.1, Eq. invM and the restricted variants after it; ILU(0) and its reuse
// within a time step, Sec. 4.2).
//
// One CTA per subdomain.  A_k = R_k J R_k^T keeps the couplings between cells of
// the box and drops the rest.  In the natural order of the box (x fastest, u before
// v) the radius-2 stencil couples cell (i, j) to earlier cells at (i-1,j), (i-2,j),
// (i-1,j-1), (i,j-1), (i+1,j-1), (i,j-2) only, so every cell of wavefront level
// l = i + 2j depends on levels < l alone: the factorization and both triangular
// sweeps run level by level, all cells of a level in parallel.
//
// ILU(0) is formed blockwise on the 2x2 (u, v) blocks: with the full 2x2 pattern on
// every stencil offset, point ILU(0) in u-before-v order and block ILU(0) drop the
// same updates, so both give the same preconditioner (L unit block-lower, U block-
// upper with pivot blocks D).  Stored per cell: the 6 lower blocks of L, D^-1, and
// the 6 upper blocks of U (52 values, zero where the neighbour is outside the box).
#include "acac_internal.cuh"

namespace acac {

template <typename T> struct V2 { T x, y; };
template <> struct __align__(16) V2<double> { double x, y; };
template <> struct __align__(8) V2<float> { float x, y; };

__device__ __forceinline__ int level_jmin(int l, int W) {
    const int t = l - W + 2;
    return t > 0 ? t / 2 : 0;
}

// Global cell of box-local (i, j).
__device__ __forceinline__ int box_cell(const Geom& g, const SubInfo& sd, int i, int j) {
    int gx = sd.ox + i, gy = sd.oy + j;
    if (gx < 0) gx += g.nx; else if (gx >= g.nx) gx -= g.nx;
    if (gy < 0) gy += g.ny; else if (gy >= g.ny) gy -= g.ny;
    return gy * g.nx + gx;
}

// Address of coefficient q of box cell (i, j) in the level-major storage.
__device__ __forceinline__ long long coef_addr(const SubInfo& sd, const int* lo, int i, int j, int q) {
    const int l = i + 2 * j;
    const int cnt = lo[l + 1] - lo[l];
    const int t = j - level_jmin(l, sd.W);
    return sd.coef_base + (long long)lo[l] * NCOEF + (long long)q * cnt + t;
}

template <typename T>
__device__ __forceinline__ void mul22(const T* a, const T* b, T* c) {
    c[0] = a[0] * b[0] + a[1] * b[2];
    c[1] = a[0] * b[1] + a[1] * b[3];
    c[2] = a[2] * b[0] + a[3] * b[2];
    c[3] = a[2] * b[1] + a[3] * b[3];
}

// ---------------------------------------------------------------- factorization
template <typename T>
__global__ void ras_factor_kernel(Geom g, const SubInfo* __restrict__ subs, const int* __restrict__ lev_off,
                                  const T* __restrict__ J, T* coef, int* flags) {
    const SubInfo sd = subs[blockIdx.x];
    const int* lo = lev_off + sd.lev_base;
    const int N = g.N;
    int bad = 0;
    for (int l = 0; l < sd.nlev; ++l) {
        const int cnt = lo[l + 1] - lo[l];
        const int jmin = level_jmin(l, sd.W);
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int j = jmin + t, i = l - 2 * j;
            const int gc = box_cell(g, sd, i, j);
            T A[NSLOT][4];
#pragma unroll
            for (int s = 0; s < NSLOT; ++s) {
                const int ii = i + slot_dx(s), jj = j + slot_dy(s);
                const bool in = ii >= 0 && ii < sd.W && jj >= 0 && jj < sd.H;
#pragma unroll
                for (int e = 0; e < 4; ++e) A[s][e] = in ? J[(size_t)(s * 4 + e) * N + gc] : (T)0;
            }
            const long long base = (long long)lo[l] * NCOEF + sd.coef_base;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const int dx1 = lower_dx(a), dy1 = lower_dy(a);
                const int ki = i + dx1, kj = j + dy1;
                T L[4] = {0, 0, 0, 0};
                if (ki >= 0 && ki < sd.W && kj >= 0 && kj < sd.H) {
                    T Dk[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) Dk[e] = coef[coef_addr(sd, lo, ki, kj, 24 + e)];
                    mul22(A[slot_of(dx1, dy1)], Dk, L);
#pragma unroll
                    for (int b = 0; b < 6; ++b) {
                        const int s2 = slot_of(dx1 + upper_dx(b), dy1 + upper_dy(b));
                        if (s2 >= 0) {
                            T U[4], P[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) U[e] = coef[coef_addr(sd, lo, ki, kj, 28 + 4 * b + e)];
                            mul22(L, U, P);
#pragma unroll
                            for (int e = 0; e < 4; ++e) A[s2][e] -= P[e];
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) coef[base + (long long)(4 * a + e) * cnt + t] = L[e];
            }
            const T* D = A[0];
            const T det = D[0] * D[3] - D[1] * D[2];
            if (!(det != (T)0) || !isfinite((double)det)) bad = 1;
            const T id = (T)1 / det;
            coef[base + (long long)24 * cnt + t] = D[3] * id;
            coef[base + (long long)25 * cnt + t] = -D[1] * id;
            coef[base + (long long)26 * cnt + t] = -D[2] * id;
            coef[base + (long long)27 * cnt + t] = D[0] * id;
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                const int s = slot_of(upper_dx(b), upper_dy(b));
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    coef[base + (long long)(28 + 4 * b + e) * cnt + t] = A[s][e];
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(flags, 4);
}

template <typename T>
cudaError_t launch_ras_factor(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off,
                              const T* J, T* coef, int threads, int* flags, cudaStream_t s) {
    ras_factor_kernel<T><<<nsub, threads, 0, s>>>(g, subs, lev_off, J, coef, flags);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- apply
// z = sum_k E_k inv(L_k U_k) R_k r with E_k the restricted (left-RAS) or full
// (AS, right-RAS) extension and R_k the full (left-RAS, AS) or restricted
// (right-RAS) restriction.  The box vector lives in a zero-padded (W+4)x(H+4)
// array (shared memory when it fits, else the subdomain's global scratch).
template <typename T>
__global__ void ras_apply_kernel(Geom g, const SubInfo* __restrict__ subs, const int* __restrict__ lev_off,
                                 const T* __restrict__ coef, const T* __restrict__ r, T* __restrict__ z,
                                 int ras_type, T* gscratch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SubInfo sd = subs[blockIdx.x];
    const int* lo = lev_off + sd.lev_base;
    const int N = g.N;
    const int PW = sd.W + 4, PH = sd.H + 4;
    V2<T>* yv = gscratch ? reinterpret_cast<V2<T>*>(gscratch) + sd.vec_base
                         : reinterpret_cast<V2<T>*>(smem_raw);
    for (int idx = threadIdx.x; idx < PW * PH; idx += blockDim.x) yv[idx] = V2<T>{(T)0, (T)0};
    __syncthreads();
    for (int idx = threadIdx.x; idx < sd.W * sd.H; idx += blockDim.x) {
        const int i = idx % sd.W, j = idx / sd.W;
        const int gc = box_cell(g, sd, i, j);
        const bool own = i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1;
        V2<T> val{r[gc], r[N + gc]};
        if (ras_type == ACAC_RAS_RIGHT && !own) val = V2<T>{(T)0, (T)0};
        yv[(j + 2) * PW + i + 2] = val;
    }
    __syncthreads();
    // forward: y_c -= sum_lower L_c,o y_{c+o}
    for (int l = 0; l < sd.nlev; ++l) {
        const int cnt = lo[l + 1] - lo[l];
        const int jmin = level_jmin(l, sd.W);
        const T* cf = coef + sd.coef_base + (long long)lo[l] * NCOEF;
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int j = jmin + t, i = l - 2 * j;
            const int pc = (j + 2) * PW + i + 2;
            V2<T> a = yv[pc];
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                const V2<T> nb = yv[pc + lower_dy(b) * PW + lower_dx(b)];
                const T l0 = cf[(4 * b + 0) * cnt + t], l1 = cf[(4 * b + 1) * cnt + t];
                const T l2 = cf[(4 * b + 2) * cnt + t], l3 = cf[(4 * b + 3) * cnt + t];
                a.x -= l0 * nb.x + l1 * nb.y;
                a.y -= l2 * nb.x + l3 * nb.y;
            }
            yv[pc] = a;
        }
        __syncthreads();
    }
    // backward: y_c = D^-1 (y_c - sum_upper U_c,o y_{c+o})
    for (int l = sd.nlev - 1; l >= 0; --l) {
        const int cnt = lo[l + 1] - lo[l];
        const int jmin = level_jmin(l, sd.W);
        const T* cf = coef + sd.coef_base + (long long)lo[l] * NCOEF;
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int j = jmin + t, i = l - 2 * j;
            const int pc = (j + 2) * PW + i + 2;
            V2<T> a = yv[pc];
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                const V2<T> nb = yv[pc + upper_dy(b) * PW + upper_dx(b)];
                const T u0 = cf[(28 + 4 * b + 0) * cnt + t], u1 = cf[(28 + 4 * b + 1) * cnt + t];
                const T u2 = cf[(28 + 4 * b + 2) * cnt + t], u3 = cf[(28 + 4 * b + 3) * cnt + t];
                a.x -= u0 * nb.x + u1 * nb.y;
                a.y -= u2 * nb.x + u3 * nb.y;
            }
            const T d0 = cf[24 * cnt + t], d1 = cf[25 * cnt + t], d2 = cf[26 * cnt + t], d3 = cf[27 * cnt + t];
            yv[pc] = V2<T>{d0 * a.x + d1 * a.y, d2 * a.x + d3 * a.y};
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < sd.W * sd.H; idx += blockDim.x) {
        const int i = idx % sd.W, j = idx / sd.W;
        const bool own = i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1;
        const int gc = box_cell(g, sd, i, j);
        const V2<T> val = yv[(j + 2) * PW + i + 2];
        if (ras_type == ACAC_RAS_LEFT) {
            if (own) { z[gc] = val.x; z[N + gc] = val.y; }
        } else {
            atomicAdd(&z[gc], val.x);
            atomicAdd(&z[N + gc], val.y);
        }
    }
}

template <typename T>
cudaError_t launch_ras_apply(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off,
                             const T* coef, const T* r, T* z, int ras_type, int threads,
                             size_t smem_bytes, T* gscratch, cudaStream_t s) {
    static bool attr_set[2] = {false, false};
    const int which = sizeof(T) == 8 ? 0 : 1;
    if (!gscratch && smem_bytes > 48 * 1024 && !attr_set[which]) {
        cudaError_t e = cudaFuncSetAttribute(ras_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[which] = true;
    }
    if (ras_type != ACAC_RAS_LEFT) {
        cudaError_t e = cudaMemsetAsync(z, 0, sizeof(T) * 2 * (size_t)g.N, s);
        if (e != cudaSuccess) return e;
    }
    ras_apply_kernel<T><<<nsub, threads, gscratch ? 0 : smem_bytes, s>>>(g, subs, lev_off, coef, r, z,
                                                                         ras_type, gscratch);
    return cudaGetLastError();
}

#define INST(T)                                                                                    \
    template cudaError_t launch_ras_factor<T>(const Geom&, int, const SubInfo*, const int*, const T*, \
                                              T*, int, int*, cudaStream_t);                         \
    template cudaError_t launch_ras_apply<T>(const Geom&, int, const SubInfo*, const int*, const T*, \
                                             const T*, T*, int, int, size_t, T*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace acac
