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
#include <atomic>
#include <mutex>

#include "acac_internal.cuh"

namespace acac {

// Raises a kernel's dynamic shared-memory limit to at least `bytes`; `done` caches the
// largest limit set so far.  Several host threads (the members of an ensemble) may
// launch the same kernel at once.
static std::mutex g_attr_mu;
static cudaError_t ensure_smem_limit(const void* func, size_t bytes, std::atomic<size_t>* done) {
    if (bytes <= done->load(std::memory_order_acquire)) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (bytes <= done->load(std::memory_order_relaxed)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done->store(bytes, std::memory_order_release);
    return e;
}

template <typename T> struct V2 { T x, y; };
template <> struct __align__(16) V2<double> { double x, y; };
template <> struct __align__(8) V2<float> { float x, y; };

__device__ __forceinline__ int level_jmin(int l, int W) {
    const int t = l - W + 2;
    return t > 0 ? t / 2 : 0;
}

// (i + dx, j + dy) inside a W x H box, for a cell (i, j) inside it: with dx, dy known at
// compile time only the sides the offset can cross are tested.
__device__ __forceinline__ bool in_box(int i, int j, int dx, int dy, int W, int H) {
    return (dx >= 0 || i + dx >= 0) && (dx <= 0 || i + dx < W) && (dy >= 0 || j + dy >= 0) && (dy <= 0 || j + dy < H);
}

// Global cell of box-local (i, j).
__device__ __forceinline__ int box_cell(const Geom& g, const SubInfo& sd, int i, int j) {
    int gx = sd.ox + i, gy = sd.oy + j;
    if (gx < 0) gx += g.nx; else if (gx >= g.nx) gx -= g.nx;
    if (gy < 0) gy += g.ny; else if (gy >= g.ny) gy -= g.ny;
    return gy * g.nx + gx;
}

// Coefficient storage of one level with cnt cells (offset lo[l] * NCOEF in the
// subdomain): a forward block of cnt records [L blocks q=0..5, row-major 2x2; 4 pad]
// and then a backward block of cnt records [D^-1 (4) | U blocks q=0..5 (24)], each
// record CREC values.  A record per cell keeps one thread's coefficients contiguous
// (wide shared loads, no per-coefficient address arithmetic); CREC = 28 makes the
// records of neighbouring threads fall into distinct shared-memory banks.
// ---------------------------------------------------------------- factorization
// Block ILU(0) row by row in wavefront order.  Row c: for every lower neighbour k in
// increasing natural order, L_ck = A_ck D_k^-1 and A_cj -= L_ck U_kj for every upper
// block U_kj of row k whose column j is in the pattern of row c; then D_c = A_cc.
// Both steps act on one block row at a time, so two threads share a cell, thread rr
// owning row rr of every 2x2 block; D_c^-1 needs both rows (one shuffle).
//
// The records of the last RING levels (every lower neighbour lies 1..4 levels back)
// are kept in shared memory for the neighbour lookups; the Jacobian rows of the next
// level are loaded into registers while the current level is computed.
constexpr int FACTOR_RING = 5;

// The factorization reads the Jacobian rows of a box's cells in wavefront order.  From
// the stencil-diagonal storage those are 26 (2D) or 50 (3D) scattered values per row (at
// 2048^2 the factorization read 9x its data in whole DRAM sectors), so the rows are first
// repacked into one record per box cell, in the factor's order: record (box cells before
// the box) + lo[level] + position, holding row 0 (slots x 2) then row 1.  One thread per
// grid cell reads its values coalesced and writes the record of every box that contains
// the cell (rec_of lists them, -1 unused).
template <typename T, int DIM>
__global__ void __launch_bounds__(256) repack_kernel(int N, const T* __restrict__ J, const int* __restrict__ rec_of,
                                                     T* __restrict__ Jp, Members mb) {
    constexpr int NS = nslot<DIM>(), NR = rec_per_cell<DIM>();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int mem = blockIdx.y;
    if (c >= N || member_off(mb, mem)) return;
    J += (size_t)mem * mb.js;
    Jp += (size_t)mem * mb.jps;
    T out[4 * NS];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int e = 0; e < 4; ++e) out[(e >> 1) * 2 * NS + 2 * s + (e & 1)] = J[(size_t)(s * 4 + e) * N + c];
    constexpr int PER = 16 / sizeof(T);          // values per 16-byte store (records are 16-byte aligned)
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const int rec = rec_of[(size_t)NR * c + q];
        if (rec < 0) continue;
        uint4* dst = reinterpret_cast<uint4*>(Jp + (size_t)rec * (4 * NS));
#pragma unroll
        for (int k = 0; k < 4 * NS / PER; ++k) dst[k] = pack16(&out[k * PER]);
    }
}

template <typename T>
cudaError_t launch_repack(const Geom& g, const T* J, const int* rec_of, T* Jp, cudaStream_t s, const Members& mb) {
    const dim3 grid((g.N + 255) / 256, mb.count);
    if (g.dim == 3) repack_kernel<T, 3><<<grid, 256, 0, s>>>(g.N, J, rec_of, Jp, mb);
    else repack_kernel<T, 2><<<grid, 256, 0, s>>>(g.N, J, rec_of, Jp, mb);
    return cudaGetLastError();
}

template <typename T>
__device__ __forceinline__ void fetch_rows(const Geom& g, const SubInfo& sd, const int* lo, const T* __restrict__ J,
                                           int packed, int l, int m, int rr, T (&dst)[NSLOT][2]) {
    const int cnt = lo[l + 1] - lo[l];
    if (m >= cnt) return;
    const int j = level_jmin(l, sd.W) + m, i = l - 2 * j;
    if (packed) {
        const T* src = J + ((size_t)(sd.coef_base / NCOEF) + lo[l] + m) * (4 * NSLOT) + rr * 2 * NSLOT;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            V2<T> v{(T)0, (T)0};
            if (in_box(i, j, slot_dx(s), slot_dy(s), sd.W, sd.H)) v = *reinterpret_cast<const V2<T>*>(src + 2 * s);
            dst[s][0] = v.x;
            dst[s][1] = v.y;
        }
        return;
    }
    const int gc = box_cell(g, sd, i, j);
    const size_t N = (size_t)g.N;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        const int ii = i + slot_dx(s), jj = j + slot_dy(s);
        const bool in = ii >= 0 && ii < sd.W && jj >= 0 && jj < sd.H;
        dst[s][0] = in ? J[(size_t)(s * 4 + 2 * rr) * N + gc] : (T)0;
        dst[s][1] = in ? J[(size_t)(s * 4 + 2 * rr + 1) * N + gc] : (T)0;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) ras_factor_kernel(Geom g, const SubInfo* __restrict__ subs,
                                                         const int* __restrict__ lev_off, const T* __restrict__ J,
                                                         int packed, T* __restrict__ coef, int ring_cells,
                                                         int* flags, Members mb) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int mem = blockIdx.y;
    if (member_off(mb, mem)) return;
    J += (size_t)mem * (packed ? mb.jps : mb.js);
    coef += (size_t)mem * mb.cfs;
    flags += mem;
    const SubInfo sd = subs[blockIdx.x];
    int* lo = reinterpret_cast<int*>(smem_raw);
    const int lev_words = (sd.nlev + 1 + 3) & ~3;
    T* ring = reinterpret_cast<T*>(smem_raw + sizeof(int) * ((lev_words + 3) & ~3));
    for (int l = threadIdx.x; l <= sd.nlev; l += blockDim.x) lo[l] = lev_off[sd.lev_base + l];
    __syncthreads();
    const int m = threadIdx.x >> 1, rr = threadIdx.x & 1;
    const int W = sd.W;
    int bad = 0;
    T Jn[NSLOT][2];
    fetch_rows<T>(g, sd, lo, J, packed, 0, m, rr, Jn);
    // ring slots (element offsets) of the levels l, l-1 .. l-4, rotated by one per level (the
    // slot of level l is l mod FACTOR_RING), and the first rows of those levels
    const int rstride = ring_cells * CREC;
    int sl0 = 0, sl1 = 4 * rstride, sl2 = 3 * rstride, sl3 = 2 * rstride, sl4 = rstride;
    for (int l = 0; l < sd.nlev; ++l) {
        T A[NSLOT][2];
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) { A[s][0] = Jn[s][0]; A[s][1] = Jn[s][1]; }
        if (l + 1 < sd.nlev) fetch_rows<T>(g, sd, lo, J, packed, l + 1, m, rr, Jn);
        const int cnt = lo[l + 1] - lo[l];
        const int jm0 = level_jmin(l, W), jm1 = level_jmin(l - 1, W), jm2 = level_jmin(l - 2, W);
        const int jm3 = level_jmin(l - 3, W), jm4 = level_jmin(l - 4, W);
        const int j = jm0 + m, i = l - 2 * j;
        const bool act = m < cnt;
        T* fw = coef + sd.coef_base + (long long)lo[l] * NCOEF + (long long)m * CREC;
        T* bw = fw + (long long)cnt * CREC;
        T* rb = ring + sl0 + m * CREC;
        if (act) {
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const int dx1 = lower_dx(a), dy1 = lower_dy(a);
                const int d = -(dx1 + 2 * dy1);           // the neighbour's level is l - d (1..4)
                T L0 = (T)0, L1 = (T)0;
                if (in_box(i, j, dx1, dy1, W, sd.H)) {
                    const int sb = d == 1 ? sl1 : d == 2 ? sl2 : d == 3 ? sl3 : sl4;
                    const int jb = d == 1 ? jm1 : d == 2 ? jm2 : d == 3 ? jm3 : jm4;
                    const T* kr = ring + sb + (j + dy1 - jb) * CREC;
                    const T* As = A[slot_of(dx1, dy1)];
                    const V2<T> p0 = *reinterpret_cast<const V2<T>*>(kr);       // kr[0], kr[1]
                    const V2<T> p1 = *reinterpret_cast<const V2<T>*>(kr + 2);   // kr[2], kr[3]
                    L0 = As[0] * p0.x + As[1] * p1.x;
                    L1 = As[0] * p0.y + As[1] * p1.y;
#pragma unroll
                    for (int b = 0; b < 6; ++b) {
                        const int s2 = slot_of(dx1 + upper_dx(b), dy1 + upper_dy(b));
                        if (s2 >= 0) {
                            const V2<T> u0 = *reinterpret_cast<const V2<T>*>(kr + 4 + 4 * b);   // U[0], U[1]
                            const V2<T> u1 = *reinterpret_cast<const V2<T>*>(kr + 6 + 4 * b);   // U[2], U[3]
                            A[s2][0] = fma(-L1, u1.x, fma(-L0, u0.x, A[s2][0]));
                            A[s2][1] = fma(-L1, u1.y, fma(-L0, u0.y, A[s2][1]));
                        }
                    }
                }
                *reinterpret_cast<V2<T>*>(fw + 4 * a + 2 * rr) = V2<T>{L0, L1};
            }
            *reinterpret_cast<V2<T>*>(fw + 24 + 2 * rr) = V2<T>{(T)0, (T)0};
        }
        // pivot block D = A[0]: row rr here, the other row in the partner lane
        const T o0 = __shfl_xor_sync(0xffffffffu, A[0][0], 1);
        const T o1 = __shfl_xor_sync(0xffffffffu, A[0][1], 1);
        if (act) {
            const T d00 = rr ? o0 : A[0][0], d01 = rr ? o1 : A[0][1];
            const T d10 = rr ? A[0][0] : o0, d11 = rr ? A[0][1] : o1;
            const T det = d00 * d11 - d01 * d10;
            if (!(det != (T)0) || !isfinite((double)det)) bad = 1;
            const T id = (T)1 / det;
            const T i0 = rr ? -d10 * id : d11 * id;    // row rr of D^-1
            const T i1 = rr ? d00 * id : -d01 * id;
            *reinterpret_cast<V2<T>*>(bw + 2 * rr) = V2<T>{i0, i1};
            *reinterpret_cast<V2<T>*>(rb + 2 * rr) = V2<T>{i0, i1};
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                const int sx = slot_of(upper_dx(b), upper_dy(b));
                *reinterpret_cast<V2<T>*>(bw + 4 + 4 * b + 2 * rr) = V2<T>{A[sx][0], A[sx][1]};
                *reinterpret_cast<V2<T>*>(rb + 4 + 4 * b + 2 * rr) = V2<T>{A[sx][0], A[sx][1]};
            }
        }
        __syncthreads();
        // level l+1 takes the slot of l-4
        const int t = sl4;
        sl4 = sl3; sl3 = sl2; sl2 = sl1; sl1 = sl0; sl0 = t;
    }
    if (bad) atomicOr(flags, 4);
}

template <typename T>
cudaError_t launch_ras_factor(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off,
                              const T* J, int packed, T* coef, int threads, int ring_cells, size_t smem_bytes,
                              int* flags, cudaStream_t s, const Members& mb) {
    static std::atomic<size_t> attr_bytes{0};
    if (smem_bytes > 48 * 1024) {
        cudaError_t e = ensure_smem_limit((const void*)ras_factor_kernel<T>, smem_bytes, &attr_bytes);
        if (e != cudaSuccess) return e;
    }
    ras_factor_kernel<T><<<dim3(nsub, mb.count), threads, smem_bytes, s>>>(g, subs, lev_off, J, packed, coef,
                                                                          ring_cells, flags, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- apply
// z = sum_k E_k inv(L_k U_k) R_k r with E_k the restricted (left-RAS) or full
// (AS, right-RAS) extension and R_k the full (left-RAS, AS) or restricted
// (right-RAS) restriction.  The box vector lives in a zero-padded (W+4)x(H+4)
// array: shared memory when it fits, else the subdomain's global scratch.
//
// The sweeps are latency bound (2 x nlev dependent levels), so the coefficients of
// each level, stored contiguously (forward part [24][cnt], backward part
// [28][cnt]), are streamed into a ring of NBUF shared-memory stages by one thread
// with cp.async.bulk (TMA) and an mbarrier per stage, NBUF levels ahead of the
// level being solved.  Stage k of the 2*nlev stages is forward level k for
// k < nlev and backward level 2*nlev-1-k after that.  Every mbarrier wait is bounded
// by the global timer; on expiry the CTA records ACAC_E_TIMEOUT in *err, drains the
// copies it issued (again bounded) and returns without writing z.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait: false after ~0.5 s without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 500000000ull) return false;
    }
}


__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Self-check of the bounded waits: the waits of the production kernels, on an mbarrier
// phase (mode 0) or a done bit (mode 1) that nothing completes.  Every lane waits; the wait
// gives up after its limit and the kernel reports it instead of hanging.
__global__ void wait_selftest_kernel(int mode, int* status) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned word;
    if (threadIdx.x == 0) {
        mbar_init(smem_addr(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        word = 0u;
    }
    __syncthreads();
    bool ok;
    if (mode == 0) {
        ok = mbar_wait_bounded(smem_addr(&bar), 0u);     // phase 0: no arrival ever comes
    } else {
        int v = 1;
        if (threadIdx.x == 0) v = wait_bit_bounded(&word, 0, 200000000ull) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, v, 0) != 0;
    }
    if (threadIdx.x == 0) *status = ok ? ACAC_OK : ACAC_E_TIMEOUT;
}

cudaError_t launch_wait_selftest(int mode, int* status, cudaStream_t s) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(mode, status);
    return cudaGetLastError();
}

// Producer / consumer pipeline.  The last warp is the producer: its lane 0 streams
// level stages into the ring (full[b] completes when a stage has landed) and reuses
// buffer b only after the consumers released it (empty[b]).  The other warps are
// the consumers: two threads per cell, thread (m, rr) solving row rr of the m-th
// cell of the level, synchronised level by level by a named barrier.
template <typename T>
__global__ void __launch_bounds__(1024) ras_apply_kernel(Geom g, const SubInfo* __restrict__ subs,
                                                        const int* __restrict__ lev_off,
                                                        const T* __restrict__ coef, const T* __restrict__ r,
                                                        T* __restrict__ z, int ras_type, T* gscratch,
                                                        RasLaunch L, int* err, Members mb, T* __restrict__ zb) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_cabort, s_pabort;   // consumer / producer gave up on a wait
    __shared__ int s_issued, s_consumed;
    const int mem = blockIdx.y;
    if (member_off(mb, mem)) return;
    coef += (size_t)mem * mb.cfs;
    r += (size_t)mem * mb.vs;
    z += (size_t)mem * mb.vs;
    if (gscratch) gscratch += (size_t)mem * mb.ss;
    if (zb) zb += (size_t)mem * mb.zs;
    err += mem;
    const SubInfo sd = subs[blockIdx.x];
    const int N = g.N;
    const int PW = ras_pitch(sd.W), PH = sd.H + 4;
    const int nlev = sd.nlev;
    const int nst = 2 * nlev;
    const int nbuf = L.nbuf;
    const int ncons = blockDim.x - 32;          // consumer threads (a multiple of 32)
    const bool producer = threadIdx.x >= ncons;
    // shared layout: full[RAS_MAXBUF] | empty[RAS_MAXBUF] | level table | stages | (box vector)
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + RAS_MAXBUF;
    int* lo = reinterpret_cast<int*>(smem_raw + 16 * RAS_MAXBUF);
    T* stages = reinterpret_cast<T*>(smem_raw + L.stage_off);
    V2<T>* yv = gscratch ? reinterpret_cast<V2<T>*>(gscratch) + sd.vec_base
                         : reinterpret_cast<V2<T>*>(smem_raw + L.vec_off);
    T* ys = reinterpret_cast<T*>(yv);        // component view: ys[2 * cell + row]
    const T* cbase = coef + sd.coef_base;

    for (int l = threadIdx.x; l <= nlev; l += blockDim.x) lo[l] = lev_off[sd.lev_base + l];
    if (threadIdx.x == 0) {
        s_cabort = 0;
        s_pabort = 0;
        s_issued = 0;
        s_consumed = 0;
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(smem_addr(&full[b]), 1);
            mbar_init(smem_addr(&empty[b]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int k) {   // stage k into buffer k % nbuf (producer lane only)
        const bool fwd = k < nlev;
        const int l = fwd ? k : nst - 1 - k;
        const int cnt = lo[l + 1] - lo[l];
        const T* src = cbase + (long long)lo[l] * NCOEF + (fwd ? 0 : (long long)cnt * CREC);
        const uint32_t bytes = (uint32_t)(CREC * cnt * sizeof(T));
        const int b = k % nbuf;
        const uint32_t bar = smem_addr(&full[b]);
        mbar_expect_tx(bar, bytes);
        bulk_g2s(smem_addr(stages + (size_t)b * L.stage_elems), src, bytes, bar);
    };
    if (threadIdx.x == ncons) {
        const int first = nbuf < nst ? nbuf : nst;
        for (int k = 0; k < first; ++k) issue(k);
        s_issued = first;
    }

    // restriction: gather r over the box (padding stays zero); loads are batched
    // GATHER at a time per thread so that their latencies overlap
    for (int idx = threadIdx.x; idx < PW * PH; idx += blockDim.x) yv[idx] = V2<T>{(T)0, (T)0};
    __syncthreads();
    constexpr int GATHER = 8;
    const int ncell = sd.W * sd.H;
    for (int base = 0; base < ncell; base += GATHER * blockDim.x) {
        V2<T> val[GATHER];
        int dst[GATHER];
#pragma unroll
        for (int q = 0; q < GATHER; ++q) {
            const int idx = base + q * blockDim.x + threadIdx.x;
            dst[q] = -1;
            if (idx < ncell) {
                const int i = idx % sd.W, j = idx / sd.W;
                const int gc = box_cell(g, sd, i, j);
                const bool own = i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1;
                val[q] = V2<T>{r[gc], r[N + gc]};
                if (ras_type == ACAC_RAS_RIGHT && !own) val[q] = V2<T>{(T)0, (T)0};
                dst[q] = (j + 2) * PW + i + 2;
            }
        }
#pragma unroll
        for (int q = 0; q < GATHER; ++q)
            if (dst[q] >= 0) yv[dst[q]] = val[q];
    }
    __syncthreads();

    if (producer) {
        if (threadIdx.x == ncons) {
            for (int k = nbuf; k < nst; ++k) {
                const int b = k % nbuf;
                if (!mbar_wait_bounded(smem_addr(&empty[b]), (uint32_t)(((k / nbuf) - 1) & 1))) {
                    s_pabort = 1;
                    break;
                }
                issue(k);
                s_issued = k + 1;
            }
        }
    } else {
        // Forward then backward sweep, one level per iteration; the stage buffer and its
        // mbarrier parity advance incrementally (no per-level division or modulo).
        const int m = threadIdx.x >> 1, rr = threadIdx.x & 1;
        const int rec_off = m * CREC + 2 * rr;          // this thread's row in a stage record
        // neighbour offsets in the padded box (cells)
        int offL[6], offU[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            offL[q] = lower_dy(q) * PW + lower_dx(q);
            offU[q] = upper_dy(q) * PW + upper_dx(q);
        }
        int k = 0, b = 0;
        uint32_t ph = 0u;
        // all consumers done with this level and with stage b; the barrier also ORs "a wait
        // gave up" over the consumers so that all of them agree
        auto finish_level = [&](bool landed) -> bool {
            uint32_t gave_up;
            asm volatile("{\n .reg .pred p, q;\n setp.eq.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n"
                         " selp.u32 %0, 1, 0, p;\n}"
                         : "=r"(gave_up) : "r"((uint32_t)landed), "r"(ncons) : "memory");
            if (gave_up) {
                if (threadIdx.x == 0) s_cabort = 1;
                return false;
            }
            if (threadIdx.x == 0) mbar_arrive(smem_addr(&empty[b]));
            if (++b == nbuf) {
                b = 0;
                ph ^= 1u;
            }
            return true;
        };
        bool aborted = false;
        for (int l = 0; l < nlev; ++l, ++k) {
            const bool landed = mbar_wait_bounded(smem_addr(&full[b]), ph);
            const int cnt = lo[l + 1] - lo[l];
            const int j = level_jmin(l, sd.W) + m, i = l - 2 * j;
            const int pc = (j + 2) * PW + i + 2;
            const T* rec = stages + (size_t)b * L.stage_elems + rec_off;
            if (m < cnt && landed) {
                // row rr: y_c -= sum_lower L_c,o y_{c+o}  (two independent chains)
                T a0 = ys[2 * pc + rr], a1 = (T)0;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const V2<T> nb = yv[pc + offL[q]];
                    const V2<T> c = *reinterpret_cast<const V2<T>*>(rec + 4 * q);
                    T& acc = q < 3 ? a0 : a1;
                    acc = fma(-c.x, nb.x, acc);
                    acc = fma(-c.y, nb.y, acc);
                }
                ys[2 * pc + rr] = a0 + a1;
            }
            if (!finish_level(landed)) {
                aborted = true;
                break;
            }
        }
        for (int l = nlev - 1; l >= 0 && !aborted; --l, ++k) {
            const bool landed = mbar_wait_bounded(smem_addr(&full[b]), ph);
            const int cnt = lo[l + 1] - lo[l];
            const int j = level_jmin(l, sd.W) + m, i = l - 2 * j;
            const int pc = (j + 2) * PW + i + 2;
            const T* rec = stages + (size_t)b * L.stage_elems + rec_off;
            const bool act = m < cnt && landed;
            // row rr of s = y_c - sum_upper U_c,o y_{c+o}; then y_c = D^-1 s
            T a0 = (T)0, a1 = (T)0;
            if (act) {
                a0 = ys[2 * pc + rr];
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    const V2<T> nb = yv[pc + offU[q]];
                    const V2<T> c = *reinterpret_cast<const V2<T>*>(rec + 4 + 4 * q);
                    T& acc = q < 3 ? a0 : a1;
                    acc = fma(-c.x, nb.x, acc);
                    acc = fma(-c.y, nb.y, acc);
                }
            }
            const T s_me = a0 + a1;
            const T s_ot = __shfl_xor_sync(0xffffffffu, s_me, 1);
            if (act) {
                const T sx = rr ? s_ot : s_me, sy = rr ? s_me : s_ot;
                const V2<T> dinv = *reinterpret_cast<const V2<T>*>(rec);
                ys[2 * pc + rr] = fma(dinv.x, sx, dinv.y * sy);
            }
            if (!finish_level(landed)) break;
        }
        if (threadIdx.x == 0) s_consumed = k;
    }
    __syncthreads();
    if (s_cabort || s_pabort) {
        // drain the copies issued but not consumed (bounded), then leave without writing z
        if (threadIdx.x == 0) {
            for (int kk = s_consumed; kk < s_issued; ++kk)
                mbar_wait_bounded(smem_addr(&full[kk % nbuf]), (uint32_t)((kk / nbuf) & 1));
            atomicOr(err, 8);
        }
        return;
    }
    // extension: left-RAS writes the owned cells of z; the additive extensions (AS,
    // right-RAS) write every box cell's values by record, summed per grid cell afterwards in
    // a fixed order (ext_gather_kernel: no atomics, the same sums run to run)
    const long long rbase = sd.coef_base / NCOEF;
    for (int idx = threadIdx.x; idx < ncell; idx += blockDim.x) {
        const int i = idx % sd.W, j = idx / sd.W;
        const bool own = i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1;
        const V2<T> val = yv[(j + 2) * PW + i + 2];
        if (ras_type == ACAC_RAS_LEFT) {
            if (own) {
                const int gc = box_cell(g, sd, i, j);
                z[gc] = val.x;
                z[N + gc] = val.y;
            }
        } else {
            const int l = i + 2 * j;
            const size_t rec = (size_t)(rbase + lo[l] + (j - level_jmin(l, sd.W)));
            *reinterpret_cast<V2<T>*>(zb + 2 * rec) = val;
        }
    }
}

// Windowed variant for boxes whose vector does not fit shared memory at two CTAs per SM
// (e.g. 132 x 132 boxes): every lower neighbour of a level-l cell lies on levels l-1..l-4
// and every upper neighbour on l+1..l+4, so shared memory keeps only the last RAS_WIN
// levels of the sweep's values, slot (l mod RAS_WIN), indexed by the row j (+2 padding
// rows on each side).  Every slot position that its level does not cover holds zero --
// the stale rows a slot's previous level left are cleared when the slot is reused, and
// the window is cleared between the sweeps -- so neighbour reads need no bounds tests.
//
// In float (PRE) the right-hand side r is gathered beforehand into every box cell's slot in
// record order (ras_gather_kernel: one coalesced pass over r, restricted to owned cells for
// right-RAS); in double the producer warp gathers it from r itself, one value per cp.async
// (the consumers' FP64 work leaves it the time).  The forward sweep writes its result in
// record order to global scratch.  Every
// stage of the ring then carries, next to the level's coefficient records, the level's
// right-hand side -- the gathered r (forward) or the forward result (backward), both
// contiguous per level -- fetched by the producer warp in 16-byte cp.async chunks that
// complete on the stage's mbarrier together with the bulk copy of the records, so the
// consumers never wait on a global load.  A backward stage is fetched only after the
// forward sweep has finished that level (a progress counter in shared memory).  Same
// barrier and bounded waits as above.
constexpr int RAS_WIN = 5;

template <typename T>
__device__ __forceinline__ void cp_async_one(uint32_t dst, const T* src, bool zero) {
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(zero ? 0 : 8)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(zero ? 0 : 4)
                     : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

template <typename T, bool PRE>
__global__ void __launch_bounds__(1024) ras_apply_win_kernel(Geom g, const SubInfo* __restrict__ subs,
                                                            const int* __restrict__ lev_off,
                                                            const T* __restrict__ coef, const T* __restrict__ r,
                                                            T* __restrict__ z, int ras_type, T* __restrict__ gscratch,
                                                            RasLaunch L, int* err, Members mb, T* __restrict__ zb) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_cabort, s_pabort;
    __shared__ int s_issued, s_consumed;
    __shared__ volatile int s_done;             // consumer steps completed (forward result in yg)
    const int mem = blockIdx.y;
    if (member_off(mb, mem)) return;
    if (zb) zb += (size_t)mem * mb.zs;
    coef += (size_t)mem * mb.cfs;
    r += (size_t)mem * (PRE ? mb.rgs : mb.vs);   // PRE: r is the gathered right-hand side
    z += (size_t)mem * mb.vs;
    gscratch += (size_t)mem * mb.ss;
    err += mem;
    const SubInfo sd = subs[blockIdx.x];
    const int N = g.N;
    const int W = sd.W, H = sd.H;
    const int nlev = sd.nlev;
    const int nst = 2 * nlev;
    const int nbuf = L.nbuf;
    const int hp = L.win_cells;                 // rows per window slot (>= H + 4)
    const int ncons = blockDim.x - 32;
    const bool producer = threadIdx.x >= ncons;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + RAS_MAXBUF;
    int* lo = reinterpret_cast<int*>(smem_raw + 16 * RAS_MAXBUF);
    T* stages = reinterpret_cast<T*>(smem_raw + L.stage_off);
    V2<T>* win = reinterpret_cast<V2<T>*>(smem_raw + L.vec_off);  // [RAS_WIN][hp]
    T* wins = reinterpret_cast<T*>(win);                            // component view
    T* yg = gscratch;                                               // forward result, by record
    const long long rbase = sd.coef_base / NCOEF;                   // records before this box
    const T* cbase = coef + sd.coef_base;

    for (int l = threadIdx.x; l <= nlev; l += blockDim.x) lo[l] = lev_off[sd.lev_base + l];
    for (int t = threadIdx.x; t < RAS_WIN * hp; t += blockDim.x) win[t] = V2<T>{(T)0, (T)0};
    if (threadIdx.x == 0) {
        s_cabort = 0;
        s_pabort = 0;
        s_issued = 0;
        s_consumed = 0;
        s_done = 0;
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(smem_addr(&full[b]), 33);   // the records' expect_tx + one arrival per producer lane
            mbar_init(smem_addr(&empty[b]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    if (producer) {
        const int lane = threadIdx.x & 31;
        for (int k = 0; k < nst; ++k) {
            const int b = k % nbuf;
            const bool fwd = k < nlev;
            const int l = fwd ? k : nst - 1 - k;
            int ok = 1;
            if (lane == 0) {
                if (k >= nbuf) ok = mbar_wait_bounded(smem_addr(&empty[b]), (uint32_t)(((k / nbuf) - 1) & 1)) ? 1 : 0;
                if (ok && !fwd) {
                    // the forward result of level l must be in the scratch: wait (bounded) for step l
                    if (s_done <= l) {
                        const uint64_t t0 = global_ns();
                        while (s_done <= l) {
                            if (s_cabort || global_ns() - t0 > 500000000ull) {
                                ok = 0;
                                break;
                            }
                        }
                    }
                    __threadfence_block();
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) s_pabort = 1;
                break;
            }
            __syncwarp();
            const int cnt = lo[l + 1] - lo[l];
            T* st = stages + (size_t)b * L.stage_elems;
            const uint32_t bar = smem_addr(&full[b]);
            if (lane == 0) {
                const T* src = cbase + (long long)lo[l] * NCOEF + (fwd ? 0 : (long long)cnt * CREC);
                const uint32_t bytes = (uint32_t)(CREC * cnt * sizeof(T));
                mbar_expect_tx(bar, bytes);
                bulk_g2s(smem_addr(st), src, bytes, bar);
            }
            // the level's right-hand side (r gathered per box cell, or the forward result), two
            // values per cell from element 2 (rbase + lo[l]) on, copied in 16-byte chunks from the
            // chunk boundary below it (the consumers skip the offset)
            T* sv = st + L.stage_vec;
            constexpr int U = 16 / (int)sizeof(T);
            if (PRE || !fwd) {
                const T* srcv = fwd ? r : yg;
                const long long e0 = 2 * (rbase + lo[l]);
                const long long a = e0 & ~(long long)(U - 1);
                const int nch = (int)((e0 - a + 2 * cnt + U - 1) / U);
                for (int c = lane; c < nch; c += 32) cp_async16(smem_addr(sv + c * U), srcv + a + (long long)c * U);
            } else {
                // r straight from the global vector, one value per cp.async, at the stage's
                // chunk offset of the level (the consumers skip it either way)
                const int voff = (int)((2 * (rbase + lo[l])) & (U - 1));
                const int jmin = level_jmin(l, W);
                const bool right = ras_type == ACAC_RAS_RIGHT;
                for (int e = lane; e < 2 * cnt; e += 32) {
                    const int m = e >> 1, rr = e & 1;
                    const int j = jmin + m, i = l - 2 * j;
                    const bool zero = right && !(i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1);
                    cp_async_one(smem_addr(sv + voff + e), r + (size_t)rr * N + box_cell(g, sd, i, j), zero);
                }
            }
            cp_async_arrive_noinc(bar);
            if (lane == 0) s_issued = k + 1;
        }
    } else {
        // Forward then backward sweep, one level per iteration.  The stage buffer and its
        // mbarrier parity advance incrementally, and the window slots of the levels l, l -+ 1,
        // .., l -+ 4 (own, n1..n4, in V2 elements past the two padding rows) rotate by one
        // per level: the bookkeeping of a level is a handful of integer operations.
        const int m = threadIdx.x >> 1, rr = threadIdx.x & 1;
        const int rec_off = m * CREC + 2 * rr;          // this thread's row in a stage record
        int b = 0;
        uint32_t ph = 0u;
        int k = 0;
        bool aborted = false;
        auto next_stage = [&]() {
            if (++b == nbuf) {
                b = 0;
                ph ^= 1u;
            }
        };
        // barrier over the consumers that also ORs "a wait gave up"; then release the stage
        auto finish_level = [&](bool landed, bool fwd_done) -> bool {
            uint32_t gave_up;
            asm volatile("{\n .reg .pred p, q;\n setp.eq.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n"
                         " selp.u32 %0, 1, 0, p;\n}"
                         : "=r"(gave_up) : "r"((uint32_t)landed), "r"(ncons) : "memory");
            if (gave_up) {
                if (threadIdx.x == 0) s_cabort = 1;
                return false;
            }
            if (threadIdx.x == 0) {
                // the backward sweep starts at the last level, whose right-hand side is the
                // forward sweep's last result: the producer needs the whole forward result
                // before its first backward stage, so the count is published once, after the
                // last forward level (a fence per level would sit on every level's path)
                if (fwd_done && k + 1 == nlev) {
                    __threadfence_block();   // the forward results in the scratch before the count
                    s_done = k + 1;
                }
                mbar_arrive(smem_addr(&empty[b]));
            }
            return true;
        };
        {   // forward: levels 0 .. nlev-1; slots of l-1 .. l-4 are 4, 3, 2, 1 at l = 0
            int own = 2, n1 = 4 * hp + 2, n2 = 3 * hp + 2, n3 = 2 * hp + 2, n4 = hp + 2;
            for (int l = 0; l < nlev; ++l, ++k) {
                const bool landed = mbar_wait_bounded(smem_addr(&full[b]), ph);
                const int cnt = lo[l + 1] - lo[l];
                const int jmin = level_jmin(l, W);
                const int j = jmin + m;
                const T* st = stages + (size_t)b * L.stage_elems;
                const bool act = m < cnt && landed;
                // clear the rows the slot's previous level (l - 5) covered below this level's
                if (l >= RAS_WIN && m < 3 && rr == 0) {
                    const int jz = level_jmin(l - RAS_WIN, W) + m;
                    if (jz < jmin) win[own + jz] = V2<T>{(T)0, (T)0};
                }
                if (act) {
                    const T* rec = st + rec_off;
                    const int voff = (int)((2 * (rbase + lo[l])) & (16 / (int)sizeof(T) - 1));
                    T a0 = st[L.stage_vec + voff + 2 * m + rr], a1 = (T)0;
                    const int off[6] = {n4 + j - 2, n3 + j - 1, n2 + j - 1, n1 + j - 1, n2 + j, n1 + j};
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const V2<T> nb = win[off[q]];
                        const V2<T> c = *reinterpret_cast<const V2<T>*>(rec + 4 * q);
                        T& acc = q < 3 ? a0 : a1;
                        acc = fma(-c.x, nb.x, acc);
                        acc = fma(-c.y, nb.y, acc);
                    }
                    const T y = a0 + a1;
                    wins[2 * (own + j) + rr] = y;
                    yg[2 * (size_t)(rbase + lo[l] + m) + rr] = y;
                }
                if (!finish_level(landed, true)) {
                    aborted = true;
                    break;
                }
                next_stage();
                // rotate the slots: level l+1 takes the slot of l-4
                const int t = n4;
                n4 = n3; n3 = n2; n2 = n1; n1 = own; own = t;
            }
        }
        if (!aborted) {
            // between the sweeps: clear the window (the backward sweep reads only its own
            // results and zeros), then start from the last level, whose slot comes first
            for (int t = threadIdx.x; t < RAS_WIN * hp; t += ncons) win[t] = V2<T>{(T)0, (T)0};
            asm volatile("bar.sync 1, %0;" ::"r"(ncons) : "memory");
            auto jmax_of = [&](int l) { const int t = l >> 1; return t < H - 1 ? t : H - 1; };
            // slots of l, l+1 .. l+4: 0, 1 .. 4 (any fixed assignment works after the clear)
            int own = 2, n1 = hp + 2, n2 = 2 * hp + 2, n3 = 3 * hp + 2, n4 = 4 * hp + 2;
            for (int l = nlev - 1; l >= 0; --l, ++k) {
                const bool landed = mbar_wait_bounded(smem_addr(&full[b]), ph);
                const int cnt = lo[l + 1] - lo[l];
                const int jmin = level_jmin(l, W);
                const int j = jmin + m, i = l - 2 * j;
                const T* st = stages + (size_t)b * L.stage_elems;
                const bool act = m < cnt && landed;
                // clear the rows the slot's previous level (l + 5) covered above this level's
                if (l + RAS_WIN < nlev && m < 3 && rr == 0) {
                    const int jz = jmax_of(l) + 1 + m;
                    if (jz <= jmax_of(l + RAS_WIN)) win[own + jz] = V2<T>{(T)0, (T)0};
                }
                T a0 = (T)0, a1 = (T)0;
                const T* rec = st + rec_off;
                if (act) {
                    const int voff = (int)((2 * (rbase + lo[l])) & (16 / (int)sizeof(T) - 1));
                    a0 = st[L.stage_vec + voff + 2 * m + rr];
                    const int off[6] = {n1 + j, n2 + j, n1 + j + 1, n2 + j + 1, n3 + j + 1, n4 + j + 2};
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const V2<T> nb = win[off[q]];
                        const V2<T> c = *reinterpret_cast<const V2<T>*>(rec + 4 + 4 * q);
                        T& acc = q < 3 ? a0 : a1;
                        acc = fma(-c.x, nb.x, acc);
                        acc = fma(-c.y, nb.y, acc);
                    }
                }
                const T s_me = a0 + a1;
                const T s_ot = __shfl_xor_sync(0xffffffffu, s_me, 1);
                if (act) {
                    const T sx = rr ? s_ot : s_me, sy = rr ? s_me : s_ot;
                    const V2<T> dinv = *reinterpret_cast<const V2<T>*>(rec);
                    const T zc = fma(dinv.x, sx, dinv.y * sy);
                    wins[2 * (own + j) + rr] = zc;
                    if (ras_type == ACAC_RAS_LEFT) {
                        if (i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1)
                            z[(size_t)rr * N + box_cell(g, sd, i, j)] = zc;
                    } else {
                        zb[2 * (size_t)(rbase + lo[l] + m) + rr] = zc;   // summed by ext_gather_kernel
                    }
                }
                if (!finish_level(landed, false)) break;
                next_stage();
                // level l-1 takes the slot of l+4
                const int t = n4;
                n4 = n3; n3 = n2; n2 = n1; n1 = own; own = t;
            }
        }
        if (threadIdx.x == 0) s_consumed = k;
    }
    __syncthreads();
    if (s_cabort || s_pabort) {
        if (threadIdx.x == 0) {
            for (int kk = s_consumed; kk < s_issued; ++kk)
                mbar_wait_bounded(smem_addr(&full[kk % nbuf]), (uint32_t)((kk / nbuf) & 1));
            atomicOr(err, 8);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) ras_gather_kernel(int N, const T* __restrict__ r, const int* __restrict__ rec_of,
                                                         const unsigned char* __restrict__ own_of, int right,
                                                         T* __restrict__ rg, Members mb) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int mem = blockIdx.y;
    if (c >= N || member_off(mb, mem)) return;
    r += (size_t)mem * mb.vs;
    rg += (size_t)mem * mb.rgs;
    const V2<T> val{r[c], r[N + c]};
    const int oq = own_of[c];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int rec = rec_of[4 * (size_t)c + q];
        if (rec < 0) break;
        *reinterpret_cast<V2<T>*>(rg + 2 * (size_t)rec) = (right && q != oq) ? V2<T>{(T)0, (T)0} : val;
    }
}

template <typename T>
cudaError_t launch_ras_gather(const Geom& g, const T* r, const int* rec_of, const unsigned char* own_of,
                              int ras_type, T* rg, cudaStream_t s, const Members& mb) {
    ras_gather_kernel<T><<<dim3((g.N + 255) / 256, mb.count), 256, 0, s>>>(
        g.N, r, rec_of, own_of, ras_type == ACAC_RAS_RIGHT ? 1 : 0, rg, mb);
    return cudaGetLastError();
}

// The additive extensions (AS, right-RAS): z at grid cell c = the sum of the values of its
// box cells (rec_of[rpc c + q], q in increasing order, -1 ends the list), written by record
// into zb by the apply kernels.  A fixed order: the same sums run to run.
template <typename T, int RPC>
__global__ void __launch_bounds__(256) ext_gather_kernel(int N, const int* __restrict__ rec_of,
                                                         const T* __restrict__ zb, T* __restrict__ z, Members mb) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int mem = blockIdx.y;
    if (c >= N || member_off(mb, mem)) return;
    zb += (size_t)mem * mb.zs;
    z += (size_t)mem * mb.vs;
    T sx = (T)0, sy = (T)0;
#pragma unroll
    for (int q = 0; q < RPC; ++q) {
        const int rec = rec_of[(size_t)RPC * c + q];
        if (rec < 0) break;
        const V2<T> v = *reinterpret_cast<const V2<T>*>(zb + 2 * (size_t)rec);
        sx += v.x;
        sy += v.y;
    }
    z[c] = sx;
    z[N + c] = sy;
}

template <typename T>
cudaError_t launch_ext_gather(const Geom& g, const int* rec_of, const T* zb, T* z, cudaStream_t s,
                              const Members& mb) {
    const dim3 grid((g.N + 255) / 256, mb.count);
    if (g.dim == 3) ext_gather_kernel<T, 8><<<grid, 256, 0, s>>>(g.N, rec_of, zb, z, mb);
    else ext_gather_kernel<T, 4><<<grid, 256, 0, s>>>(g.N, rec_of, zb, z, mb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ras_apply(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off,
                             const T* coef, const T* r, T* z, int ras_type, int threads,
                             const RasLaunch& L, T* gscratch, const T* rg, int* err, cudaStream_t s,
                             const Members& mb, const int* rec_of, T* zb) {
    static std::atomic<size_t> attr_bytes{0};
    const dim3 grid(nsub, mb.count);
    const bool additive = ras_type != ACAC_RAS_LEFT;
    if (additive && (!rec_of || !zb)) return cudaErrorInvalidValue;
    if (!L.window) {
        cudaError_t e = ensure_smem_limit((const void*)ras_apply_kernel<T>, L.smem_bytes, &attr_bytes);
        if (e != cudaSuccess) return e;
    }
    if (L.window) {
        static std::atomic<size_t> win_bytes{0}, win_bytes_pre{0};
        cudaError_t e = rg ? ensure_smem_limit((const void*)ras_apply_win_kernel<T, true>, L.smem_bytes, &win_bytes_pre)
                           : ensure_smem_limit((const void*)ras_apply_win_kernel<T, false>, L.smem_bytes, &win_bytes);
        if (e != cudaSuccess) return e;
        // float: r gathered beforehand (the producer keeps up only with contiguous copies);
        // double: the producer gathers r itself (the consumers' FP64 work leaves it time)
        if (rg)
            ras_apply_win_kernel<T, true><<<grid, threads, L.smem_bytes, s>>>(g, subs, lev_off, coef, rg, z, ras_type,
                                                                              gscratch, L, err, mb, zb);
        else
            ras_apply_win_kernel<T, false><<<grid, threads, L.smem_bytes, s>>>(g, subs, lev_off, coef, r, z, ras_type,
                                                                               gscratch, L, err, mb, zb);
    } else {
        ras_apply_kernel<T><<<grid, threads, L.smem_bytes, s>>>(g, subs, lev_off, coef, r, z, ras_type, gscratch, L,
                                                                err, mb, zb);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !additive) return e;
    return launch_ext_gather<T>(g, rec_of, zb, z, s, mb);
}


// ================================================================ 3D
// Same factorization and sweeps on 3D boxes: wavefront level l = i + 2j + 3k, 12 lower and
// 12 upper 2x2 blocks per cell, records of CREC3 values.  The cells of each level come from
// a per-subdomain list (packed i | j << 10 | k << 20, in level order) and a map from the
// box-local cell index to its position in its level.  One CTA per subdomain, two threads per
// cell (one per block row); records are read from global memory.
__device__ __forceinline__ void unpack3(int p, int& i, int& j, int& k) {
    i = p & 1023;
    j = (p >> 10) & 1023;
    k = p >> 20;
}
__device__ __forceinline__ int box_cell3(const Geom& g, const SubInfo& sd, int i, int j, int k) {
    const bool per = g.bc == ACAC_BC_PERIODIC;
    const int gx = wrap_or_clamp(sd.ox + i, g.nx, per), gy = wrap_or_clamp(sd.oy + j, g.ny, per);
    const int gz = wrap_or_clamp(sd.oz + k, g.nz, per);
    return (gz * g.ny + gy) * g.nx + gx;
}

template <typename T>
__global__ void __launch_bounds__(512) ras_factor3_kernel(Geom g, const SubInfo* __restrict__ subs,
                                                          const int* __restrict__ lev_off, const int* __restrict__ cells,
                                                          const int* __restrict__ pos, const T* __restrict__ J,
                                                          int packed, T* coef, int* flags, Members mb) {
    const int mem = blockIdx.y;
    if (member_off(mb, mem)) return;
    J += (size_t)mem * (packed ? mb.jps : mb.js);
    coef += (size_t)mem * mb.cfs;
    flags += mem;
    const SubInfo sd = subs[blockIdx.x];
    const int* lo = lev_off + sd.lev_base;
    const int* cl = cells + sd.cell_base;
    const int* ps = pos + sd.cell_base;
    const size_t N = (size_t)g.N;
    const int rr = threadIdx.x & 1;
    int bad = 0;
    for (int l = 0; l < sd.nlev; ++l) {
        const int cnt = lo[l + 1] - lo[l];
        T* lvl = coef + sd.coef_base + (long long)lo[l] * NCOEF3;
        for (int m = threadIdx.x >> 1; m < (cnt + 15) / 16 * 16; m += blockDim.x >> 1) {
            const bool act = m < cnt;
            int i = 0, j = 0, k = 0;
            if (act) unpack3(cl[lo[l] + m], i, j, k);
            T A[NSLOT3][2];
            if (act) {
                // row rr of the cell: its record (packed) or the stencil-diagonal storage
                const int gc = box_cell3(g, sd, i, j, k);
                const T* rec = J + ((size_t)(sd.coef_base / NCOEF3) + lo[l] + m) * (4 * NSLOT3) + rr * 2 * NSLOT3;
#pragma unroll
                for (int s = 0; s < NSLOT3; ++s) {
                    const int ii = i + s3_dx(s), jj = j + s3_dy(s), kk = k + s3_dz(s);
                    const bool in = ii >= 0 && ii < sd.W && jj >= 0 && jj < sd.H && kk >= 0 && kk < sd.D;
                    const T v0 = packed ? rec[2 * s] : J[(size_t)(s * 4 + 2 * rr) * N + gc];
                    const T v1 = packed ? rec[2 * s + 1] : J[(size_t)(s * 4 + 2 * rr + 1) * N + gc];
                    A[s][0] = in ? v0 : (T)0;
                    A[s][1] = in ? v1 : (T)0;
                }
            } else {
#pragma unroll
                for (int s = 0; s < NSLOT3; ++s) { A[s][0] = (T)0; A[s][1] = (T)0; }
            }
            T* fw = lvl + (long long)m * CREC3;
            T* bw = lvl + (long long)(cnt + m) * CREC3;
            if (act) {
#pragma unroll
                for (int a = 0; a < 12; ++a) {
                    const int dx1 = l3_dx(a), dy1 = l3_dy(a), dz1 = l3_dz(a);
                    const int ki = i + dx1, kj = j + dy1, kk = k + dz1;
                    T L0 = (T)0, L1 = (T)0;
                    if (ki >= 0 && ki < sd.W && kj >= 0 && kj < sd.H && kk >= 0 && kk < sd.D) {
                        const int lk = l + dx1 + 2 * dy1 + 3 * dz1;
                        const int tk = ps[(kk * sd.H + kj) * sd.W + ki];
                        const int ck = lo[lk + 1] - lo[lk];
                        const T* kr = coef + sd.coef_base + (long long)lo[lk] * NCOEF3 + (long long)(ck + tk) * CREC3;
                        const T* As = A[slot3_of(dx1, dy1, dz1)];
                        L0 = As[0] * kr[0] + As[1] * kr[2];
                        L1 = As[0] * kr[1] + As[1] * kr[3];
#pragma unroll
                        for (int b = 0; b < 12; ++b) {
                            const int s2 = slot3_of(dx1 + u3_dx(b), dy1 + u3_dy(b), dz1 + u3_dz(b));
                            if (s2 >= 0) {
                                const T* U = kr + 4 + 4 * b;
                                A[s2][0] = fma(-L1, U[2], fma(-L0, U[0], A[s2][0]));
                                A[s2][1] = fma(-L1, U[3], fma(-L0, U[1], A[s2][1]));
                            }
                        }
                    }
                    fw[4 * a + 2 * rr] = L0;
                    fw[4 * a + 2 * rr + 1] = L1;
                }
                fw[48 + 2 * rr] = (T)0;
                fw[49 + 2 * rr] = (T)0;
            }
            const T o0 = __shfl_xor_sync(0xffffffffu, A[0][0], 1);
            const T o1 = __shfl_xor_sync(0xffffffffu, A[0][1], 1);
            if (act) {
                const T d00 = rr ? o0 : A[0][0], d01 = rr ? o1 : A[0][1];
                const T d10 = rr ? A[0][0] : o0, d11 = rr ? A[0][1] : o1;
                const T det = d00 * d11 - d01 * d10;
                if (!(det != (T)0) || !isfinite((double)det)) bad = 1;
                const T id = (T)1 / det;
                bw[2 * rr] = rr ? -d10 * id : d11 * id;
                bw[2 * rr + 1] = rr ? d00 * id : -d01 * id;
#pragma unroll
                for (int b = 0; b < 12; ++b) {
                    const int s = slot3_of(u3_dx(b), u3_dy(b), u3_dz(b));
                    bw[4 + 4 * b + 2 * rr] = A[s][0];
                    bw[4 + 4 * b + 2 * rr + 1] = A[s][1];
                }
            }
        }
        __syncthreads();
    }
    if (bad) atomicOr(flags, 4);
}

template <typename T>
__global__ void __launch_bounds__(1024) ras_apply3_kernel(Geom g, const SubInfo* __restrict__ subs,
                                                         const int* __restrict__ lev_off, const int* __restrict__ cells,
                                                         const T* __restrict__ coef, const T* __restrict__ r,
                                                         T* __restrict__ z, int ras_type, T* gscratch, RasLaunch L,
                                                         int* err, Members mb, T* __restrict__ zb) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ int s_cabort, s_pabort;
    __shared__ int s_issued, s_consumed;
    const int mem = blockIdx.y;
    if (member_off(mb, mem)) return;
    if (zb) zb += (size_t)mem * mb.zs;
    coef += (size_t)mem * mb.cfs;
    r += (size_t)mem * mb.vs;
    z += (size_t)mem * mb.vs;
    if (gscratch) gscratch += (size_t)mem * mb.ss;
    err += mem;
    const SubInfo sd = subs[blockIdx.x];
    const int* cl = cells + sd.cell_base;
    const int N = g.N;
    const int PW = ras3_pitch(sd.W, sizeof(T)), PH = sd.H + 4, PD = sd.D + 4;
    const int plane = PW * PH;
    const int nlev = sd.nlev;
    const int nst = 2 * nlev;
    const int nbuf = L.nbuf;
    const int ncons = blockDim.x - 32;
    const bool producer = threadIdx.x >= ncons;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
    uint64_t* empty = full + RAS_MAXBUF;
    int* lo = reinterpret_cast<int*>(smem_raw + 16 * RAS_MAXBUF);
    T* stages = reinterpret_cast<T*>(smem_raw + L.stage_off);
    V2<T>* yv = gscratch ? reinterpret_cast<V2<T>*>(gscratch) + sd.vec_base
                         : reinterpret_cast<V2<T>*>(smem_raw + L.vec_off);
    T* ys = reinterpret_cast<T*>(yv);
    const T* cbase = coef + sd.coef_base;

    for (int l = threadIdx.x; l <= nlev; l += blockDim.x) lo[l] = lev_off[sd.lev_base + l];
    if (threadIdx.x == 0) {
        s_cabort = 0;
        s_pabort = 0;
        s_issued = 0;
        s_consumed = 0;
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(smem_addr(&full[b]), 1);
            mbar_init(smem_addr(&empty[b]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int k) {   // stage k: the level's forward or backward records
        const bool fwd = k < nlev;
        const int l = fwd ? k : nst - 1 - k;
        const int cnt = lo[l + 1] - lo[l];
        const T* src = cbase + (long long)lo[l] * NCOEF3 + (fwd ? 0 : (long long)cnt * CREC3);
        const uint32_t bytes = (uint32_t)(CREC3 * cnt * sizeof(T));
        const int b = k % nbuf;
        const uint32_t bar = smem_addr(&full[b]);
        mbar_expect_tx(bar, bytes);
        bulk_g2s(smem_addr(stages + (size_t)b * L.stage_elems), src, bytes, bar);
    };
    if (threadIdx.x == ncons) {
        const int first = nbuf < nst ? nbuf : nst;
        for (int k = 0; k < first; ++k) issue(k);
        s_issued = first;
    }
    // restriction: the box with a zero padding of 2
    for (int idx = threadIdx.x; idx < plane * PD; idx += blockDim.x) yv[idx] = V2<T>{(T)0, (T)0};
    __syncthreads();
    const int ncell = sd.W * sd.H * sd.D;
    for (int idx = threadIdx.x; idx < ncell; idx += blockDim.x) {
        const int i = idx % sd.W, j = (idx / sd.W) % sd.H, k = idx / (sd.W * sd.H);
        const int gc = box_cell3(g, sd, i, j, k);
        const bool own = i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1 &&
                         k >= sd.own_z0 && k < sd.own_z1;
        V2<T> val{r[gc], r[N + gc]};
        if (ras_type == ACAC_RAS_RIGHT && !own) val = V2<T>{(T)0, (T)0};
        yv[((k + 2) * PH + j + 2) * PW + i + 2] = val;
    }
    __syncthreads();

    if (producer) {
        if (threadIdx.x == ncons) {
            for (int k = nbuf; k < nst; ++k) {
                const int b = k % nbuf;
                if (!mbar_wait_bounded(smem_addr(&empty[b]), (uint32_t)(((k / nbuf) - 1) & 1))) {
                    s_pabort = 1;
                    break;
                }
                issue(k);
                s_issued = k + 1;
            }
        }
    } else {
        const int m = threadIdx.x >> 1, rr = threadIdx.x & 1;
        // packed cell of position m of the next stage's level, prefetched a stage ahead
        auto cell_at = [&](int kk) -> int {
            if (kk >= nst) return 0;
            const int l = kk < nlev ? kk : nst - 1 - kk;
            return m < lo[l + 1] - lo[l] ? cl[lo[l] + m] : 0;
        };
        int pk = cell_at(0);
        int k = 0;
        for (; k < nst; ++k) {
            const int b = k % nbuf;
            const int cur = pk;
            pk = cell_at(k + 1);
            const bool landed = mbar_wait_bounded(smem_addr(&full[b]), (uint32_t)((k / nbuf) & 1));
            const bool fwd = k < nlev;
            const int l = fwd ? k : nst - 1 - k;
            const int cnt = lo[l + 1] - lo[l];
            const bool act = m < cnt && landed;
            int i = 0, j = 0, kz = 0;
            unpack3(cur, i, j, kz);
            const int pc = ((kz + 2) * PH + j + 2) * PW + i + 2;
            const T* rec = stages + (size_t)b * L.stage_elems + (size_t)m * CREC3 + (fwd ? 0 : 4) + 2 * rr;
            T a0 = (T)0, a1 = (T)0;
            if (act) {
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const int off = fwd ? (l3_dz(q) * plane + l3_dy(q) * PW + l3_dx(q))
                                        : (u3_dz(q) * plane + u3_dy(q) * PW + u3_dx(q));
                    const V2<T> nb = yv[pc + off];
                    T& acc = q < 6 ? a0 : a1;
                    acc = fma(rec[4 * q], nb.x, acc);
                    acc = fma(rec[4 * q + 1], nb.y, acc);
                }
            }
            const T s_me = (act ? ys[2 * pc + rr] : (T)0) - (a0 + a1);
            if (fwd) {
                if (act) ys[2 * pc + rr] = s_me;
            } else {
                const T s_ot = __shfl_xor_sync(0xffffffffu, s_me, 1);
                if (act) {
                    const T* di = stages + (size_t)b * L.stage_elems + (size_t)m * CREC3 + 2 * rr;
                    const T sx = rr ? s_ot : s_me, sy = rr ? s_me : s_ot;
                    ys[2 * pc + rr] = fma(di[0], sx, di[1] * sy);
                }
            }
            uint32_t gave_up;
            asm volatile("{\n .reg .pred p, q;\n setp.eq.u32 q, %1, 0;\n bar.red.or.pred p, 1, %2, q;\n"
                         " selp.u32 %0, 1, 0, p;\n}"
                         : "=r"(gave_up) : "r"((uint32_t)landed), "r"(ncons) : "memory");
            if (gave_up) {
                if (threadIdx.x == 0) s_cabort = 1;
                break;
            }
            if (threadIdx.x == 0) mbar_arrive(smem_addr(&empty[b]));
        }
        if (threadIdx.x == 0) s_consumed = k;
    }
    __syncthreads();
    if (s_cabort || s_pabort) {
        if (threadIdx.x == 0) {
            for (int kk = s_consumed; kk < s_issued; ++kk)
                mbar_wait_bounded(smem_addr(&full[kk % nbuf]), (uint32_t)((kk / nbuf) & 1));
            atomicOr(err, 8);
        }
        return;
    }
    if (ras_type == ACAC_RAS_LEFT) {
        for (int idx = threadIdx.x; idx < ncell; idx += blockDim.x) {
            const int i = idx % sd.W, j = (idx / sd.W) % sd.H, k = idx / (sd.W * sd.H);
            if (!(i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1 && k >= sd.own_z0 &&
                  k < sd.own_z1))
                continue;
            const int gc = box_cell3(g, sd, i, j, k);
            const V2<T> val = yv[((k + 2) * PH + j + 2) * PW + i + 2];
            z[gc] = val.x;
            z[N + gc] = val.y;
        }
    } else {
        // additive extensions: every box cell's values by record (the level-ordered cell list),
        // summed per grid cell in a fixed order by ext_gather_kernel
        const long long rbase = sd.coef_base / NCOEF3;
        for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
            const int pk = cl[t];
            const int i = pk & 1023, j = (pk >> 10) & 1023, k = pk >> 20;
            *reinterpret_cast<V2<T>*>(zb + 2 * (size_t)(rbase + t)) = yv[((k + 2) * PH + j + 2) * PW + i + 2];
        }
    }
}

template <typename T>
cudaError_t launch_ras_factor3(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off, const int* cells,
                               const int* pos, const T* J, int packed, T* coef, int threads, int* flags,
                               cudaStream_t s, const Members& mb) {
    ras_factor3_kernel<T><<<dim3(nsub, mb.count), threads, 0, s>>>(g, subs, lev_off, cells, pos, J, packed, coef,
                                                                   flags, mb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ras_apply3(const Geom& g, int nsub, const SubInfo* subs, const int* lev_off, const int* cells,
                              const T* coef, const T* r, T* z, int ras_type, const RasLaunch& L, T* gscratch,
                              int* err, cudaStream_t s, const Members& mb, const int* rec_of, T* zb) {
    static std::atomic<size_t> attr_bytes{0};
    const bool additive = ras_type != ACAC_RAS_LEFT;
    if (additive && (!rec_of || !zb)) return cudaErrorInvalidValue;
    {
        cudaError_t e = ensure_smem_limit((const void*)ras_apply3_kernel<T>, L.smem_bytes, &attr_bytes);
        if (e != cudaSuccess) return e;
    }
    ras_apply3_kernel<T><<<dim3(nsub, mb.count), L.threads, L.smem_bytes, s>>>(g, subs, lev_off, cells, coef, r, z,
                                                                              ras_type, gscratch, L, err, mb, zb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !additive) return e;
    return launch_ext_gather<T>(g, rec_of, zb, z, s, mb);
}

#define INST(T)                                                                                    \
    template cudaError_t launch_repack<T>(const Geom&, const T*, const int*, T*, cudaStream_t, const Members&); \
    template cudaError_t launch_ras_factor<T>(const Geom&, int, const SubInfo*, const int*, const T*, \
                                              int, T*, int, int, size_t, int*, cudaStream_t, const Members&); \
    template cudaError_t launch_ras_gather<T>(const Geom&, const T*, const int*, const unsigned char*, \
                                              int, T*, cudaStream_t, const Members&);                   \
    template cudaError_t launch_ras_apply<T>(const Geom&, int, const SubInfo*, const int*, const T*, \
                                             const T*, T*, int, int, const RasLaunch&, T*, const T*, int*, \
                                             cudaStream_t, const Members&, const int*, T*);           \
    template cudaError_t launch_ext_gather<T>(const Geom&, const int*, const T*, T*, cudaStream_t,     \
                                              const Members&);                                        \
    template cudaError_t launch_ras_factor3<T>(const Geom&, int, const SubInfo*, const int*, const int*,    \
                                               const int*, const T*, int, T*, int, int*, cudaStream_t,      \
                                               const Members&);                                             \
    template cudaError_t launch_ras_apply3<T>(const Geom&, int, const SubInfo*, const int*, const int*,     \
                                              const T*, const T*, T*, int, const RasLaunch&, T*, int*,     \
                                              cudaStream_t, const Members&, const int*, T*);
INST(double)
INST(float)
#undef INST

}  // namespace acac
