// Subdomain solves with fill for the Schwarz preconditioner (Sec. 3.1, and the
// subdomain-solver comparison of Sec. 4.2, Table 2): ILU(1), ILU(2) and exact LU of the
// box matrices A_k, beside the fill-free wavefront ILU(0) of ras.cu.
//
// Every box matrix is stored by 2x2 blocks on a pattern over the box's cells in natural
// order (x fastest, then y, then z).  Since every 2x2 block of A_k is full, the level of
// fill of a point entry is that of its pair of cells, and the point factorization in
// u-before-v order keeps whole blocks: the block IKJ elimination on the cell pattern
// gives the same factors.  The pattern is built on the host once per box shape:
//   ILU(p): levels of fill, lev = 0 on the stencil, lev(i,j) = min over the eliminated
//           k < i of lev(i,k) + lev(k,j) + 1, entries of level <= p kept;
//   LU:     every entry of the profile (fill never leaves the row's first stencil
//           column on the left, nor a column's first stencil row above), a superset of
//           the fill of the exact factorization, which keeps its values exact.
// The factorization runs in dataflow order (rows in natural order over the warps, each
// step waiting for the row it reads); the two triangular sweeps run level by level over
// the rows' dependency levels, one CTA per box and one warp per row of a level.
#include <algorithm>
#include <functional>
#include <queue>

#include "acac_internal.cuh"

namespace acac {

// ---------------------------------------------------------------- host: symbolic
namespace {
struct Off { int dx, dy, dz; };

std::vector<Off> stencil(int dim) {
    std::vector<Off> o;
    if (dim == 2)
        for (int s = 0; s < NSLOT; ++s) o.push_back({slot_dx(s), slot_dy(s), 0});
    else
        for (int s = 0; s < NSLOT3; ++s) o.push_back({s3_dx(s), s3_dy(s), s3_dz(s)});
    return o;
}

// rows' dependency levels: lev[i] = 1 + max lev over deps(i), in the given visiting order
void levels_of(int n, const std::vector<int>& lev, std::vector<int>& ptr, std::vector<int>& rows) {
    int nl = 0;
    for (int i = 0; i < n; ++i) nl = std::max(nl, lev[i] + 1);
    ptr.assign(nl + 1, 0);
    for (int i = 0; i < n; ++i) ptr[lev[i] + 1]++;
    for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
    rows.assign(n, 0);
    std::vector<int> fillp(ptr.begin(), ptr.end() - 1);
    for (int i = 0; i < n; ++i) rows[fillp[lev[i]]++] = i;
}
}  // namespace

SparseShape build_sparse_shape(int dim, int W, int H, int D, int fill) {
    SparseShape S;
    S.dim = dim;
    S.W = W;
    S.H = H;
    S.D = dim == 3 ? D : 1;
    const int n = W * H * S.D;
    S.n = n;
    const std::vector<Off> st = stencil(dim);
    const int ns = (int)st.size();
    auto nb = [&](int c, const Off& o) {
        const int i = c % W, j = (c / W) % H, k = c / (W * H);
        const int ii = i + o.dx, jj = j + o.dy, kk = k + o.dz;
        if (ii < 0 || ii >= W || jj < 0 || jj >= H || kk < 0 || kk >= S.D) return -1;
        return ii + W * (jj + H * kk);
    };
    std::vector<std::vector<int>> cols(n);
    if (fill < 0) {
        // LU: the profile.  lo[i] = first stencil column of row i; the upper part of row
        // i holds the columns j >= i whose first stencil row lo[j] (the structure is
        // symmetric) is at most i: up to hi[i] = max{j : lo[j] <= i}
        std::vector<int> lo(n), best(n, -1), hi(n);
        for (int c = 0; c < n; ++c) {
            int m = c;
            for (const Off& o : st) {
                const int t = nb(c, o);
                if (t >= 0) m = std::min(m, t);
            }
            lo[c] = m;
            best[m] = std::max(best[m], c);
        }
        int run = -1;
        for (int i = 0; i < n; ++i) {
            run = std::max(run, best[i]);
            hi[i] = std::max(run, i);
        }
        for (int i = 0; i < n; ++i)
            for (int j = lo[i]; j <= hi[i]; ++j) cols[i].push_back(j);
    } else {
        // ILU(fill): levels of fill, eliminating row i's entries left of the diagonal in
        // increasing column order (fill entries created on the way included)
        const int INF = 1 << 29;
        std::vector<std::vector<std::pair<int, int>>> rows(n);   // (column, level), sorted
        std::vector<int> lev(n, INF);
        std::vector<int> touched;
        for (int i = 0; i < n; ++i) {
            touched.clear();
            std::priority_queue<int, std::vector<int>, std::greater<int>> pq;
            for (const Off& o : st) {
                const int t = nb(i, o);
                if (t < 0) continue;
                lev[t] = 0;
                touched.push_back(t);
                if (t < i) pq.push(t);
            }
            int last = -1;
            while (!pq.empty()) {
                const int k = pq.top();
                pq.pop();
                if (k == last) continue;
                last = k;
                const int lik = lev[k];
                for (const auto& e : rows[k]) {
                    if (e.first <= k) continue;
                    const int cand = lik + e.second + 1;
                    if (cand > fill || cand >= lev[e.first]) continue;
                    if (lev[e.first] == INF) {
                        touched.push_back(e.first);
                        if (e.first < i) pq.push(e.first);
                    }
                    lev[e.first] = cand;
                }
            }
            std::sort(touched.begin(), touched.end());
            for (int j : touched) {
                rows[i].push_back({j, lev[j]});
                cols[i].push_back(j);
                lev[j] = INF;
            }
        }
    }
    S.ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) S.ptr[i + 1] = S.ptr[i] + (int)cols[i].size();
    S.col.reserve(S.ptr[n]);
    S.diag.assign(n, -1);
    S.band = 0;
    for (int i = 0; i < n; ++i) {
        for (int j : cols[i]) {
            if (j == i) S.diag[i] = (int)S.col.size();
            S.band = std::max(S.band, std::abs(j - i));
            S.col.push_back(j);
        }
    }
    S.slot_pos.assign((size_t)n * ns, -1);
    for (int i = 0; i < n; ++i)
        for (int s = 0; s < ns; ++s) {
            const int t = nb(i, st[s]);
            if (t < 0) continue;
            const auto b = S.col.begin() + S.ptr[i], e = S.col.begin() + S.ptr[i + 1];
            const auto it = std::lower_bound(b, e, t);
            S.slot_pos[(size_t)i * ns + s] = (int)(it - S.col.begin());
        }
    // dependency levels: forward through L (columns < i), backward through U (> i)
    std::vector<int> fl(n, 0), bl(n, 0);
    for (int i = 0; i < n; ++i)
        for (int p = S.ptr[i]; p < S.diag[i]; ++p) fl[i] = std::max(fl[i], fl[S.col[p]] + 1);
    for (int i = n - 1; i >= 0; --i)
        for (int p = S.diag[i] + 1; p < S.ptr[i + 1]; ++p) bl[i] = std::max(bl[i], bl[S.col[p]] + 1);
    levels_of(n, fl, S.flev_ptr, S.flev_rows);
    levels_of(n, bl, S.blev_ptr, S.blev_rows);
    S.contig = 1;
    for (int i = 0; i < n && S.contig; ++i)
        if (S.col[S.ptr[i + 1] - 1] - S.col[S.ptr[i]] != S.ptr[i + 1] - S.ptr[i] - 1) S.contig = 0;
    return S;
}

// ---------------------------------------------------------------- device
namespace {

__device__ __forceinline__ int global_cell(const Geom& g, const SubInfo& sd, int c, int& i, int& j, int& k) {
    i = c % sd.W;
    j = (c / sd.W) % sd.H;
    k = c / (sd.W * sd.H);
    const bool per = g.bc == ACAC_BC_PERIODIC;
    const int gx = wrap_or_clamp(sd.ox + i, g.nx, per), gy = wrap_or_clamp(sd.oy + j, g.ny, per);
    const int gz = g.dim == 3 ? wrap_or_clamp(sd.oz + k, g.nz, per) : 0;
    return (gz * g.ny + gy) * g.nx + gx;
}

__device__ __forceinline__ bool owned(const SubInfo& sd, int i, int j, int k) {
    return i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1 && k >= sd.own_z0 && k < sd.own_z1;
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_d(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

template <typename T, int DIM>
__global__ void __launch_bounds__(256) sparse_init_kernel(Geom g, const SubInfo* __restrict__ subs,
                                                          const SparseBox* __restrict__ boxes,
                                                          const SparseShapeDev* __restrict__ shapes,
                                                          const T* __restrict__ J, T* __restrict__ val, Members mb) {
    const int mem = blockIdx.y;
    if (member_off(mb, mem)) return;
    J += (size_t)mem * mb.js;
    val += (size_t)mem * mb.cfs;
    const SubInfo sd = subs[blockIdx.x];
    const SparseBox bx = boxes[blockIdx.x];
    const SparseShapeDev sh = shapes[bx.shape];
    constexpr int NS = nslot<DIM>();
    const size_t N = (size_t)g.N;
    T* A = val + 4 * bx.blk_base;
    for (int c = threadIdx.x; c < sh.n; c += blockDim.x) {
        int i, j, k;
        const int gc = global_cell(g, sd, c, i, j, k);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int pos = sh.slot_pos[(size_t)c * NS + s];
            if (pos < 0) continue;
#pragma unroll
            for (int e = 0; e < 4; ++e) A[4 * (size_t)pos + e] = J[(size_t)(s * 4 + e) * N + gc];
        }
    }
}

// Block IKJ elimination of row i:
//   for k in L(i) ascending:  L_ik = A_ik D_k^-1;  A_ij -= L_ik U_kj  for j in U(k) kept in row i
//   D_i = A_ii, its inverse stored.
// Dataflow order: the warps take the rows in natural order, round robin, and a warp at
// step k first waits until row k is final (a done bit per row in shared memory, set
// after the row's values).  Rows therefore proceed concurrently wherever their
// dependencies allow -- under LU every dependency level holds a single row, yet
// consecutive rows overlap on all but their last steps and read the same rows U(k)
// at about the same time.  Every wait is bounded by the global timer; on expiry the
// block records bit 3 of *flags and stops.
// Positions: on a contiguous pattern (every row an interval of columns, as the LU
// profile is) the position of (i, j) is arithmetic; otherwise the warp's map (2 band + 1
// ints in shared memory) takes j - i + band to it, -1 where row i keeps no entry (the
// update is dropped).
template <typename T>
__global__ void __launch_bounds__(1024) sparse_factor_kernel(const SparseBox* __restrict__ boxes,
                                                             const SparseShapeDev* __restrict__ shapes,
                                                             T* val, T* dinv, int* flags, int use_map, Members mb) {
    extern __shared__ int smem[];
    const int mem = blockIdx.y;
    if (member_off(mb, mem)) return;
    val += (size_t)mem * mb.cfs;
    dinv += (size_t)mem * mb.rgs;
    flags += mem;
    const SparseBox bx = boxes[blockIdx.x];
    const SparseShapeDev sh = shapes[bx.shape];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int n = sh.n, B = sh.band, MW = 2 * B + 1;
    const int nwords = (n + 31) >> 5;
    unsigned* done = reinterpret_cast<unsigned*>(smem);
    int* map = smem + ((nwords + 3) & ~3) + (size_t)warp * MW;
    const bool contig = sh.contig != 0;
    for (int t = threadIdx.x; t < nwords; t += blockDim.x) done[t] = 0u;
    if (use_map && !contig)
        for (int t = lane; t < MW; t += 32) map[t] = -1;
    __syncthreads();
    T* A = val + 4 * bx.blk_base;
    T* Di = dinv + 4 * bx.cell_base;
    int bad = 0, timed_out = 0;
    for (int i = warp; i < n && !timed_out; i += nw) {
        const int p0 = sh.ptr[i], p1 = sh.ptr[i + 1], pd = sh.diag[i];
        const int c0 = sh.col[p0];
        if (!contig) {
            for (int p = p0 + lane; p < p1; p += 32) map[sh.col[p] - i + B] = p;
            __syncwarp();
        }
        for (int p = p0; p < pd; ++p) {
            const int k = contig ? c0 + (p - p0) : sh.col[p];
            // row k final?  Lane 0 polls (bounded) and the warp takes its result
            int ok = 1;
            if (lane == 0) {
                ok = wait_bit_bounded(done + (k >> 5), k & 31, SPARSE_WAIT_NS) ? 1 : 0;
                __threadfence_block();
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                timed_out = 1;
                break;
            }
            __syncwarp();
            __threadfence_block();
            const T* dk = Di + 4 * (size_t)k;
            const T a00 = A[4 * (size_t)p], a01 = A[4 * (size_t)p + 1];
            const T a10 = A[4 * (size_t)p + 2], a11 = A[4 * (size_t)p + 3];
            const T l00 = a00 * dk[0] + a01 * dk[2], l01 = a00 * dk[1] + a01 * dk[3];
            const T l10 = a10 * dk[0] + a11 * dk[2], l11 = a10 * dk[1] + a11 * dk[3];
            __syncwarp();
            if (lane == 0) {
                A[4 * (size_t)p] = l00;
                A[4 * (size_t)p + 1] = l01;
                A[4 * (size_t)p + 2] = l10;
                A[4 * (size_t)p + 3] = l11;
            }
            const int dk0 = sh.diag[k], u1 = sh.ptr[k + 1];
            for (int u = dk0 + 1 + lane; u < u1; u += 32) {
                int t;
                if (contig) {
                    t = p0 + (k + (u - dk0) - c0);   // column k + (u - dk0) of row i
                } else {
                    t = map[sh.col[u] - i + B];
                    if (t < 0) continue;
                }
                const T* U = A + 4 * (size_t)u;
                T* X = A + 4 * (size_t)t;
                const T u00 = U[0], u01 = U[1], u10 = U[2], u11 = U[3];
                X[0] = fma(-l01, u10, fma(-l00, u00, X[0]));
                X[1] = fma(-l01, u11, fma(-l00, u01, X[1]));
                X[2] = fma(-l11, u10, fma(-l10, u00, X[2]));
                X[3] = fma(-l11, u11, fma(-l10, u01, X[3]));
            }
            __syncwarp();
        }
        if (timed_out) break;
        if (lane == 0) {
            const T* d = A + 4 * (size_t)pd;
            const T det = d[0] * d[3] - d[1] * d[2];
            if (!(det != (T)0) || !isfinite((double)det)) bad = 1;
            const T id = (T)1 / det;
            T* o = Di + 4 * (size_t)i;
            o[0] = d[3] * id;
            o[1] = -d[1] * id;
            o[2] = -d[2] * id;
            o[3] = d[0] * id;
        }
        if (!contig) {
            for (int p = p0 + lane; p < p1; p += 32) map[sh.col[p] - i + B] = -1;
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) atomicOr(done + (i >> 5), 1u << (i & 31));
    }
    if (bad) atomicOr(flags, 4);
    if (timed_out && lane == 0) atomicOr(flags, 8);
}

// Restriction, forward sweep y_i = r_i - sum_{k<i} L_ik y_k, backward sweep
// z_i = D_i^-1 (y_i - sum_{j>i} U_ij z_j), extension; one warp per row of a level, the
// row's blocks over the lanes.
template <typename T>
__global__ void __launch_bounds__(256) sparse_apply_kernel(Geom g, const SubInfo* __restrict__ subs,
                                                           const SparseBox* __restrict__ boxes,
                                                           const SparseShapeDev* __restrict__ shapes,
                                                           const T* __restrict__ val, const T* __restrict__ dinv,
                                                           const T* __restrict__ r, T* __restrict__ z, int ras_type,
                                                           T* yscratch, int in_smem, Members mb, T* __restrict__ zb) {
    extern __shared__ __align__(16) unsigned char sraw[];
    const int mem = blockIdx.y;
    if (member_off(mb, mem)) return;
    if (zb) zb += (size_t)mem * mb.zs;
    val += (size_t)mem * mb.cfs;
    dinv += (size_t)mem * mb.rgs;
    r += (size_t)mem * mb.vs;
    z += (size_t)mem * mb.vs;
    if (yscratch) yscratch += (size_t)mem * mb.ss;
    const SubInfo sd = subs[blockIdx.x];
    const SparseBox bx = boxes[blockIdx.x];
    const SparseShapeDev sh = shapes[bx.shape];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T* y = in_smem ? reinterpret_cast<T*>(sraw) : yscratch + 2 * bx.cell_base;
    const T* A = val + 4 * bx.blk_base;
    const T* Di = dinv + 4 * bx.cell_base;
    const size_t N = (size_t)g.N;
    for (int c = threadIdx.x; c < sh.n; c += blockDim.x) {
        int i, j, k;
        const int gc = global_cell(g, sd, c, i, j, k);
        const bool keep = ras_type != ACAC_RAS_RIGHT || owned(sd, i, j, k);
        y[2 * c] = keep ? r[gc] : (T)0;
        y[2 * c + 1] = keep ? r[N + gc] : (T)0;
    }
    __syncthreads();
    __shared__ T red[2][8];
    // sum over positions [pa, pb) of row blocks times y, by the warp (lanes strided) or,
    // for a level of a single row, by the whole block (threads strided)
    auto row_dot = [&](int pa, int pb, int tid, int nt, T& s0, T& s1) {
        s0 = (T)0;
        s1 = (T)0;
        for (int p = pa + tid; p < pb; p += nt) {
            const T* a = A + 4 * (size_t)p;
            const int c = sh.col[p];
            const T y0 = y[2 * c], y1 = y[2 * c + 1];
            s0 = fma(a[1], y1, fma(a[0], y0, s0));
            s1 = fma(a[3], y1, fma(a[2], y0, s1));
        }
        s0 = warp_sum_d(s0);
        s1 = warp_sum_d(s1);
    };
    auto block_total = [&](T& s0, T& s1) {   // after row_dot over the block: total in thread 0
        if (lane == 0) {
            red[0][warp] = s0;
            red[1][warp] = s1;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s0 = (T)0;
            s1 = (T)0;
            for (int w = 0; w < nw; ++w) {
                s0 += red[0][w];
                s1 += red[1][w];
            }
        }
    };
    for (int lv = 0; lv < sh.nflev; ++lv) {
        const int q0 = sh.flev_ptr[lv], q1 = sh.flev_ptr[lv + 1];
        if (q1 - q0 == 1 && nw > 1) {
            const int i = sh.flev_rows[q0];
            T s0, s1;
            row_dot(sh.ptr[i], sh.diag[i], threadIdx.x, blockDim.x, s0, s1);
            block_total(s0, s1);
            if (threadIdx.x == 0) {
                y[2 * i] -= s0;
                y[2 * i + 1] -= s1;
            }
        } else {
            for (int q = q0 + warp; q < q1; q += nw) {
                const int i = sh.flev_rows[q];
                T s0, s1;
                row_dot(sh.ptr[i], sh.diag[i], lane, 32, s0, s1);
                if (lane == 0) {
                    y[2 * i] -= s0;
                    y[2 * i + 1] -= s1;
                }
            }
        }
        __syncthreads();
    }
    for (int lv = 0; lv < sh.nblev; ++lv) {
        const int q0 = sh.blev_ptr[lv], q1 = sh.blev_ptr[lv + 1];
        const bool whole = q1 - q0 == 1 && nw > 1;
        for (int q = q0 + (whole ? 0 : warp); q < q1; q += (whole ? 1 : nw)) {
            const int i = sh.blev_rows[q];
            T s0, s1;
            row_dot(sh.diag[i] + 1, sh.ptr[i + 1], whole ? (int)threadIdx.x : lane, whole ? (int)blockDim.x : 32, s0,
                    s1);
            if (whole) block_total(s0, s1);
            if (whole ? threadIdx.x == 0 : lane == 0) {
                const T t0 = y[2 * i] - s0, t1 = y[2 * i + 1] - s1;
                const T* d = Di + 4 * (size_t)i;
                y[2 * i] = d[0] * t0 + d[1] * t1;
                y[2 * i + 1] = d[2] * t0 + d[3] * t1;
            }
        }
        __syncthreads();
    }
    for (int c = threadIdx.x; c < sh.n; c += blockDim.x) {
        int i, j, k;
        const int gc = global_cell(g, sd, c, i, j, k);
        if (ras_type == ACAC_RAS_LEFT) {
            if (owned(sd, i, j, k)) {
                z[gc] = y[2 * c];
                z[N + gc] = y[2 * c + 1];
            }
        } else {
            // additive extensions: by box cell (natural order within the box), summed per grid
            // cell in a fixed order afterwards (launch_ext_gather)
            zb[2 * (size_t)(bx.cell_base + c)] = y[2 * c];
            zb[2 * (size_t)(bx.cell_base + c) + 1] = y[2 * c + 1];
        }
    }
}

template <typename T>
cudaError_t launch_sparse_init(const Geom& g, int nbox, const SubInfo* subs, const SparseBox* boxes,
                               const SparseShapeDev* shapes, const T* J, T* val, cudaStream_t s, const Members& mb) {
    const dim3 grid(nbox, mb.count);
    if (g.dim == 3) sparse_init_kernel<T, 3><<<grid, 256, 0, s>>>(g, subs, boxes, shapes, J, val, mb);
    else sparse_init_kernel<T, 2><<<grid, 256, 0, s>>>(g, subs, boxes, shapes, J, val, mb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sparse_factor(int nbox, const SparseBox* boxes, const SparseShapeDev* shapes, T* val, T* dinv,
                                 int* flags, int threads, size_t smem, int use_map, cudaStream_t s,
                                 const Members& mb) {
    if (threads < 32 || threads > 1024 || threads % 32) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sparse_factor_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    sparse_factor_kernel<T><<<dim3(nbox, mb.count), threads, smem, s>>>(boxes, shapes, val, dinv, flags, use_map, mb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sparse_apply(const Geom& g, int nbox, const SubInfo* subs, const SparseBox* boxes,
                                const SparseShapeDev* shapes, const T* val, const T* dinv, const T* r, T* z,
                                int ras_type, T* yscratch, int threads, size_t smem, cudaStream_t s,
                                const Members& mb, const int* rec_of, T* zb) {
    const bool additive = ras_type != ACAC_RAS_LEFT;
    if (additive && (!rec_of || !zb)) return cudaErrorInvalidValue;
    if (threads < 32 || threads > 256 || threads % 32) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sparse_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    sparse_apply_kernel<T><<<dim3(nbox, mb.count), threads, smem, s>>>(g, subs, boxes, shapes, val, dinv, r, z,
                                                                       ras_type, yscratch, smem > 0 ? 1 : 0, mb, zb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !additive) return e;
    return launch_ext_gather<T>(g, rec_of, zb, z, s, mb);
}

#define INST(T)                                                                                                   \
    template cudaError_t launch_sparse_init<T>(const Geom&, int, const SubInfo*, const SparseBox*,                 \
                                               const SparseShapeDev*, const T*, T*, cudaStream_t, const Members&); \
    template cudaError_t launch_sparse_factor<T>(int, const SparseBox*, const SparseShapeDev*, T*, T*, int*, int,  \
                                                 size_t, int, cudaStream_t, const Members&);                      \
    template cudaError_t launch_sparse_apply<T>(const Geom&, int, const SubInfo*, const SparseBox*,                \
                                                const SparseShapeDev*, const T*, const T*, const T*, T*, int, T*,  \
                                                int, size_t, cudaStream_t, const Members&, const int*, T*);
INST(double)
INST(float)
#undef INST

}  // namespace acac
