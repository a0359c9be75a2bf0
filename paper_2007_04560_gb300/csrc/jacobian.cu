// Jacobian of F (scheme NSOA-1, Sec. 2) at an iterate X1: analytic assembly into
// stencil-diagonal 2x2-block storage, the assembled product y = J w, and the
// matrix-free product y = J(X1) w from the per-cell linearisation cache.
//
// With the cache entries of cell k (c, cu, cv, Gu, Gv, du, xc; dv = du + (alpha-beta)/2):
//   dG_u(k) = du w_u + xc w_v - gamma/2 [Delta w_u](k)
//   dG_v(k) = xc w_u + dv w_v - gamma/2 [Delta w_v](k)
//   dc(k)   = cu w_u + cv w_v
//   (J w)_u(c) = w_u/dt - sum_f open_f/h_f^2 [ (dc_c+dc_n)/2 (Gu_n-Gu_c) + (c_c+c_n)/2 (dG_u(n)-dG_u(c)) ]
//   (J w)_v(c) = w_v/dt + (dc_c Gv_c + c_c dG_v(c)) / rho
#include "acac_internal.cuh"

namespace acac {

static int grid1(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < (1 << 30) ? (b < 1 ? 1 : b) : (1 << 30));
}

// ---------------------------------------------------------------- assembly
// J is written in stencil-diagonal storage, or (PACKED) straight into the records of the
// subdomain factorization (one 4 x nslot-value record per box that contains the cell,
// rec_of[REC_PER_CELL c + q]; see the repack kernel of the factorization), which skips the
// stencil-diagonal pass when nothing else reads it.
template <typename T, int DIM, bool PACKED>
__global__ void __launch_bounds__(128) assemble_kernel(Geom g, const JacK<T>* __restrict__ kp, Cache<T> C,
                                                       T* __restrict__ J, const int* __restrict__ rec_of, Members mb) {
    constexpr int NS = nslot<DIM>();
    constexpr int NF = 2 * DIM;
    const int N = g.N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (c >= N || member_off(mb, m)) return;
    const JacK<T> k = kp[m];
    C = member_cache(C, mb, m);
    J += (size_t)m * (PACKED ? mb.jps : mb.js);
    int x, y, z;
    decode_cell<DIM>(g, c, x, y, z);
    // arithmetic in the Jacobian's precision T
    const T hg = k.hg, dvshift = k.dvs;
    const T half = (T)0.5;
    T Juu[NS], Juv[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) { Juu[s] = (T)0; Juv[s] = (T)0; }
    const T cc = C.c[c], cuc = C.cu[c], cvc = C.cv[c], gc = C.Gu[c], gvc = C.Gv[c];
    const T duc = C.du[c], xcc = C.xc[c];
    const bool per = g.bc == ACAC_BC_PERIODIC;
    T lapc = (T)0;   // sum of open faces / h^2 at c
    T eih2c[NF], ehc[NF];   // 1/h^2 and 1/(2 h^2) of the open faces, 0 for closed ones
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const bool o = face_open<DIM>(g, x, y, z, f);
        eih2c[f] = o ? (sizeof(T) == 8 ? (T)face_ih2(g, f) : (T)(f < 2 ? g.ihx2f : f < 4 ? g.ihy2f : g.ihz2f)) : (T)0;
        ehc[f] = o ? face_half<T>(g, f) : (T)0;
        lapc += eih2c[f];
    }
    // Face f (weight w = 1/h^2 if open, else 0; neighbour n; ct = (c_c + c_n)/2;
    // dG = G_u(n) - G_u(c)) contributes to the u row
    //   -w/2 dG (c_u, c_v)(c)      at the centre       (mobility variation at c)
    //   -w/2 dG (c_u, c_v)(n)      at the face slot    (mobility variation at n)
    //   -w ct (du, xc)(n)          at the face slot    (pointwise part of dG_u(n))
    //   +w ct hg e2(n, f2)         at n + face f2, and -w ct hg lap(n) at the face slot
    //                              (Laplacian part of dG_u(n), lap(n) = sum_f2 e2(n, f2))
    //   +w ct (du, xc)(c)          at the centre       (pointwise part of dG_u(c))
    //   -w ct hg e(c, f2)          at c + face f2, +w ct hg lap(c) at the centre.
    // The centre terms depend on f only through S1 = sum_f w dG and W = sum_f w ct, which
    // are summed first (about half the FP64 operations of accumulating them per face).
    T S1 = (T)0, W = (T)0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        const int fx = fc_dx<DIM>(f), fy = fc_dy<DIM>(f), fz = fc_dz<DIM>(f);
        const int sf = sl_of<DIM>(fx, fy, fz);
        const int n = face_nb<DIM>(g, x, y, z, f);
        const T w = eih2c[f], hw = ehc[f];
        const T dG = C.Gu[n] - gc;
        const T wct = hw * (cc + C.c[n]);
        const T t = hw * dG;
        S1 = fma(w, dG, S1);
        W += wct;
        const int nx_ = x + fx, ny_ = y + fy, nz_ = z + fz;
        const T wcth = wct * hg;
        // lap(n); on a periodic grid every face is open and lap(n) = lap(c) (the same
        // weights summed in the same order)
        T lapn = (T)0;
#pragma unroll
        for (int f2 = 0; f2 < NF; ++f2) {
            const T e2 = face_weight<DIM, T>(g, nx_, ny_, nz_, f2);
            const int s2 = sl_of<DIM>(fx + fc_dx<DIM>(f2), fy + fc_dy<DIM>(f2), fz + fc_dz<DIM>(f2));
            Juu[s2] = fma(wcth, e2, Juu[s2]);
            if (!per) lapn += e2;
        }
        if (per) lapn = lapc;
        Juu[sf] -= fma(wct, fma(hg, lapn, C.du[n]), t * C.cu[n]);
        Juv[sf] -= fma(wct, C.xc[n], t * C.cv[n]);
    }
    Juu[0] += k.idt + fma(W, fma(hg, lapc, duc), -half * cuc * S1);
    Juv[0] += fma(W, xcc, -half * cvc * S1);
    const T hgW = hg * W;
#pragma unroll
    for (int f2 = 0; f2 < NF; ++f2) {
        const int s2 = sl_of<DIM>(fc_dx<DIM>(f2), fc_dy<DIM>(f2), fc_dz<DIM>(f2));
        Juu[s2] = fma(-hgW, eih2c[f2], Juu[s2]);
    }
    const T irho = k.irho;
    const T cgi = -cc * hg * irho;   // face entries of the v row: -c gamma/2 w / rho
    T Jvu[NS], Jvv[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        T jvu = (T)0, jvv = (T)0;
        if (s == 0) {
            jvu = (cuc * gvc + cc * xcc) * irho;
            jvv = k.idt + (cvc * gvc + cc * (duc + dvshift + hg * lapc)) * irho;
        } else if (s <= NF) {
            const int f = s - 1;   // slots 1..2*DIM are the faces
            jvv = cgi * eih2c[f];
        }
        Jvu[s] = jvu;
        Jvv[s] = jvv;
    }
    if (!PACKED) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            J[(size_t)(s * 4 + 0) * N + c] = Juu[s];
            J[(size_t)(s * 4 + 1) * N + c] = Juv[s];
            J[(size_t)(s * 4 + 2) * N + c] = Jvu[s];
            J[(size_t)(s * 4 + 3) * N + c] = Jvv[s];
        }
        return;
    }
    // record: row 0 (slots x (uu, uv)), row 1 (slots x (vu, vv))
    T out[4 * NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        out[2 * s] = Juu[s];
        out[2 * s + 1] = Juv[s];
        out[2 * NS + 2 * s] = Jvu[s];
        out[2 * NS + 2 * s + 1] = Jvv[s];
    }
    constexpr int NR = rec_per_cell<DIM>();
    constexpr int PER = 16 / sizeof(T);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const int rec = rec_of[(size_t)NR * c + q];
        if (rec < 0) continue;
        uint4* dst = reinterpret_cast<uint4*>(J + (size_t)rec * (4 * NS));
#pragma unroll
        for (int kk = 0; kk < 4 * NS / PER; ++kk) dst[kk] = pack16(&out[kk * PER]);
    }
}

template <typename T>
cudaError_t launch_assemble(const Geom& g, const JacK<T>* kp, Cache<T> cache, T* J, cudaStream_t s,
                            const int* rec_of, const Members& mb) {
    const dim3 grid(grid1(g.N, 128), mb.count);
    if (g.dim == 3) {
        if (rec_of) assemble_kernel<T, 3, true><<<grid, 128, 0, s>>>(g, kp, cache, J, rec_of, mb);
        else assemble_kernel<T, 3, false><<<grid, 128, 0, s>>>(g, kp, cache, J, nullptr, mb);
    } else {
        if (rec_of) assemble_kernel<T, 2, true><<<grid, 128, 0, s>>>(g, kp, cache, J, rec_of, mb);
        else assemble_kernel<T, 2, false><<<grid, 128, 0, s>>>(g, kp, cache, J, nullptr, mb);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- assembled product
template <typename T, int DIM>
__global__ void __launch_bounds__(256) spmv_kernel(Geom g, const T* __restrict__ J, const T* __restrict__ w,
                                                   T* __restrict__ y, Members mb) {
    const int N = g.N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (c >= N || member_off(mb, m)) return;
    J += (size_t)m * mb.js;
    w += (size_t)m * mb.vs;
    y += (size_t)m * mb.vs;
    int x, yy, zz;
    decode_cell<DIM>(g, c, x, yy, zz);
    T au = 0, av = 0;
#pragma unroll
    for (int s = 0; s < nslot<DIM>(); ++s) {
        const int n = slot_nb<DIM>(g, x, yy, zz, s);
        const T wu = w[n], wv = w[N + n];
        au = fma(J[(size_t)(s * 4 + 1) * N + c], wv, fma(J[(size_t)(s * 4 + 0) * N + c], wu, au));
        av = fma(J[(size_t)(s * 4 + 3) * N + c], wv, fma(J[(size_t)(s * 4 + 2) * N + c], wu, av));
    }
    y[c] = au;
    y[N + c] = av;
}

template <typename T>
cudaError_t launch_spmv(const Geom& g, const T* J, const T* w, T* y, cudaStream_t s, const Members& mb) {
    const dim3 grid(grid1(g.N, 256), mb.count);
    if (g.dim == 3) spmv_kernel<T, 3><<<grid, 256, 0, s>>>(g, J, w, y, mb);
    else spmv_kernel<T, 2><<<grid, 256, 0, s>>>(g, J, w, y, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- matrix-free product
// Pass 1: dG_u, dG_v, dc per cell into tmp = [dGu | dGv | dc].
template <typename T, int DIM>
__global__ void __launch_bounds__(256) jvp1_kernel(Geom g, const JacK<T>* __restrict__ kp, Cache<T> C,
                                                   const T* __restrict__ w, T* __restrict__ tmp, Members mb) {
    const int N = g.N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (c >= N || member_off(mb, m)) return;
    kp += m;
    C = member_cache(C, mb, m);
    w += (size_t)m * mb.vs;
    tmp += (size_t)m * mb.gs;
    int x, y, z;
    decode_cell<DIM>(g, c, x, y, z);
    const T wu = w[c], wv = w[N + c];
    // Laplacian per axis, (w_- + w_+ - 2 w) / h^2: a clamped (Neumann wall) neighbour is the
    // cell itself and adds nothing
    T lu = 0, lv = 0;
    if (g.iso) {
        // equal spacing: the neighbour sums first, one scaling by 1/h^2
        T nu = 0, nv = 0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int nm = face_nb<DIM>(g, x, y, z, 2 * d), np = face_nb<DIM>(g, x, y, z, 2 * d + 1);
            nu = d == 0 ? w[nm] + w[np] : nu + (w[nm] + w[np]);
            nv = d == 0 ? w[N + nm] + w[N + np] : nv + (w[N + nm] + w[N + np]);
        }
        const T ih2 = sizeof(T) == 8 ? (T)g.ihx2 : (T)g.ihx2f;
        lu = fma((T)(-2 * DIM), wu, nu) * ih2;
        lv = fma((T)(-2 * DIM), wv, nv) * ih2;
    } else {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const int nm = face_nb<DIM>(g, x, y, z, 2 * d), np = face_nb<DIM>(g, x, y, z, 2 * d + 1);
            const T ih2 = sizeof(T) == 8 ? (T)face_ih2(g, 2 * d) : (T)(d == 0 ? g.ihx2f : d == 1 ? g.ihy2f : g.ihz2f);
            lu = fma(fma((T)-2, wu, w[nm] + w[np]), ih2, lu);
            lv = fma(fma((T)-2, wv, w[N + nm] + w[N + np]), ih2, lv);
        }
    }
    const JacK<T> k = *kp;
    const T hg = k.hg;
    const T du = C.du[c], xc = C.xc[c], dv = du + k.dvs;
    tmp[c] = du * wu + xc * wv - hg * lu;
    tmp[N + c] = xc * wu + dv * wv - hg * lv;
    tmp[2 * N + c] = C.cu[c] * wu + C.cv[c] * wv;
}

template <typename T, int DIM>
__global__ void __launch_bounds__(256) jvp2_kernel(Geom g, const JacK<T>* __restrict__ kp, Cache<T> C,
                                                   const T* __restrict__ w, const T* __restrict__ tmp,
                                                   T* __restrict__ y, Members mb) {
    const int N = g.N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = blockIdx.y;
    if (c >= N || member_off(mb, m)) return;
    kp += m;
    C = member_cache(C, mb, m);
    w += (size_t)m * mb.vs;
    tmp += (size_t)m * mb.gs;
    y += (size_t)m * mb.vs;
    int x, yy, zz;
    decode_cell<DIM>(g, c, x, yy, zz);
    const T* dGu = tmp;
    const T* dGv = tmp + N;
    const T* dc = tmp + 2 * N;
    const T cc = C.c[c], gc = C.Gu[c], dgc = dGu[c], dcc = dc[c];
    T div = 0;
    if (g.iso) {
        // equal spacing: every face has the weight 1/(2 h^2), applied once to the sum
        T t = 0;
#pragma unroll
        for (int f = 0; f < 2 * DIM; ++f) {
            const int n = face_nb<DIM>(g, x, yy, zz, f);
            t = f == 0 ? (dcc + dc[n]) * (C.Gu[n] - gc) : fma(dcc + dc[n], C.Gu[n] - gc, t);
            t = fma(cc + C.c[n], dGu[n] - dgc, t);
        }
        div = face_half<T>(g, 0) * t;
    } else {
#pragma unroll
        for (int f = 0; f < 2 * DIM; ++f) {
            const int n = face_nb<DIM>(g, x, yy, zz, f);
            div = fma(face_half<T>(g, f), fma(cc + C.c[n], dGu[n] - dgc, (dcc + dc[n]) * (C.Gu[n] - gc)), div);
        }
    }
    const T idt = kp->idt, irho = kp->irho;
    y[c] = w[c] * idt - div;
    y[N + c] = w[N + c] * idt + (dcc * C.Gv[c] + cc * dGv[c]) * irho;
}

template <typename T>
cudaError_t launch_jvp_g(const Geom& g, const JacK<T>* kp, Cache<T> cache, const T* w, T* tmp, cudaStream_t s,
                         const Members& mb) {
    const dim3 grid(grid1(g.N, 256), mb.count);
    if (g.dim == 3) jvp1_kernel<T, 3><<<grid, 256, 0, s>>>(g, kp, cache, w, tmp, mb);
    else jvp1_kernel<T, 2><<<grid, 256, 0, s>>>(g, kp, cache, w, tmp, mb);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jvp_f(const Geom& g, const JacK<T>* kp, Cache<T> cache, const T* w, const T* tmp, T* y,
                         cudaStream_t s, const Members& mb) {
    const dim3 grid(grid1(g.N, 256), mb.count);
    if (g.dim == 3) jvp2_kernel<T, 3><<<grid, 256, 0, s>>>(g, kp, cache, w, tmp, y, mb);
    else jvp2_kernel<T, 2><<<grid, 256, 0, s>>>(g, kp, cache, w, tmp, y, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fused tiled product (2D)
// y = J(X1) w in one pass over a JT_X x JT_Y tile of output cells: w is staged with a
// 2-cell halo and c, G_u with a 1-cell halo in shared memory; dG_u and dc are formed on
// the 1-cell ring, dG_v on the tile; then the face fluxes.  Block coordinates give (x, y)
// without division; neighbours outside the grid are wrapped (periodic) or clamped
// (Neumann: their face weight is 0).  Algorithmic traffic: w (2), the cache (7) and y (2)
// per cell.  Each staging phase first issues all of a thread's loads into registers and
// only then uses them, so that ~30 loads per thread are in flight (the kernel is bound
// by load latency otherwise).
constexpr int JT_X = 64, JT_Y = 16, JT_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(JT_THREADS, 4) jvp_tile_kernel(Geom g, const JacK<T>* __restrict__ kp, Cache<T> C,
                                                              const T* __restrict__ w, T* __restrict__ y, Members mb) {
    constexpr int WX = JT_X + 4, WY = JT_Y + 4;     // w with halo 2
    constexpr int RX = JT_X + 2, RY = JT_Y + 2;     // ring with halo 1
    constexpr int NW = (WX * WY + JT_THREADS - 1) / JT_THREADS;
    constexpr int NR = (RX * RY + JT_THREADS - 1) / JT_THREADS;
    constexpr int NO = JT_X * JT_Y / JT_THREADS;
    __shared__ T swu[WY][WX], swv[WY][WX];
    __shared__ T sc[RY][RX], sg[RY][RX], sdg[RY][RX], sdc[RY][RX];
    __shared__ T sdgv[JT_Y][JT_X];
    const int N = g.N;
    const int m = blockIdx.z;
    if (member_off(mb, m)) return;
    kp += m;
    C = member_cache(C, mb, m);
    w += (size_t)m * mb.vs;
    y += (size_t)m * mb.vs;
    const int x0 = blockIdx.x * JT_X, y0 = blockIdx.y * JT_Y;
    const bool per = g.bc == ACAC_BC_PERIODIC;
    const int tid = threadIdx.x;
    // G_v of this thread's output cells, needed only at the end
    T gv[NO];
#pragma unroll
    for (int k = 0; k < NO; ++k) {
        const int idx = tid + k * JT_THREADS;
        const int gx = x0 + idx % JT_X, gy = y0 + idx / JT_X;
        gv[k] = (gx < g.nx && gy < g.ny) ? C.Gv[gy * g.nx + gx] : (T)0;
    }
    // phase 1: w with a 2-cell halo
    {
        T au[NW], av[NW];
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int idx = tid + k * JT_THREADS;
            au[k] = av[k] = (T)0;
            if (idx < WX * WY) {
                const int lx = idx % WX, ly = idx / WX;
                const int gx = wrap_or_clamp(x0 + lx - 2, g.nx, per), gy = wrap_or_clamp(y0 + ly - 2, g.ny, per);
                const int gc = gy * g.nx + gx;
                au[k] = w[gc];
                av[k] = w[N + gc];
            }
        }
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int idx = tid + k * JT_THREADS;
            if (idx < WX * WY) {
                swu[idx / WX][idx % WX] = au[k];
                swv[idx / WX][idx % WX] = av[k];
            }
        }
    }
    // phase 2 loads (independent of w): the cache on the 1-cell ring
    T rc[NR], rg[NR], rdu[NR], rxc[NR], rcu[NR], rcv[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int idx = tid + k * JT_THREADS;
        rc[k] = rg[k] = rdu[k] = rxc[k] = rcu[k] = rcv[k] = (T)0;
        if (idx < RX * RY) {
            const int lx = idx % RX, ly = idx / RX;
            const int cx = wrap_or_clamp(x0 + lx - 1, g.nx, per), cy = wrap_or_clamp(y0 + ly - 1, g.ny, per);
            const int gc = cy * g.nx + cx;
            rc[k] = C.c[gc];
            rg[k] = C.Gu[gc];
            rdu[k] = C.du[gc];
            rxc[k] = C.xc[gc];
            rcu[k] = C.cu[gc];
            rcv[k] = C.cv[gc];
        }
    }
    __syncthreads();
    const JacK<T> k = *kp;
    const T hg = k.hg, dvs = k.dvs;
    const T ihx2 = sizeof(T) == 8 ? (T)g.ihx2 : (T)g.ihx2f, ihy2 = sizeof(T) == 8 ? (T)g.ihy2 : (T)g.ihy2f;
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const int idx = tid + q * JT_THREADS;
        if (idx >= RX * RY) continue;
        const int lx = idx % RX, ly = idx / RX;
        const int wx = lx + 1, wy = ly + 1;             // position in the w tile
        const T wu = swu[wy][wx], wv = swv[wy][wx];
        // Laplacians with the ghost rule (clamped neighbours give zero differences)
        const T lu = (swu[wy][wx - 1] + swu[wy][wx + 1] - (T)2 * wu) * ihx2 + (swu[wy - 1][wx] + swu[wy + 1][wx] - (T)2 * wu) * ihy2;
        sc[ly][lx] = rc[q];
        sg[ly][lx] = rg[q];
        sdg[ly][lx] = rdu[q] * wu + rxc[q] * wv - hg * lu;
        sdc[ly][lx] = rcu[q] * wu + rcv[q] * wv;
        if (lx >= 1 && lx <= JT_X && ly >= 1 && ly <= JT_Y) {
            const T lv = (swv[wy][wx - 1] + swv[wy][wx + 1] - (T)2 * wv) * ihx2 + (swv[wy - 1][wx] + swv[wy + 1][wx] - (T)2 * wv) * ihy2;
            sdgv[ly - 1][lx - 1] = rxc[q] * wu + (rdu[q] + dvs) * wv - hg * lv;
        }
    }
    __syncthreads();
    const T idt = k.idt, irho = k.irho, half = (T)0.5;
#pragma unroll
    for (int q = 0; q < NO; ++q) {
        const int idx = tid + q * JT_THREADS;
        const int tx = idx % JT_X, ty = idx / JT_X;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx >= g.nx || gy >= g.ny) continue;
        const int rx = tx + 1, ry = ty + 1;
        const T cc = sc[ry][rx], gc_ = sg[ry][rx], dgc = sdg[ry][rx], dcc = sdc[ry][rx];
        T div = (T)0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const int nx_ = rx + face_dx(f), ny_ = ry + face_dy(f);
            const T wf = face_w<T>(g, gx, gy, f);
            div += wf * (half * (dcc + sdc[ny_][nx_]) * (sg[ny_][nx_] - gc_) + half * (cc + sc[ny_][nx_]) * (sdg[ny_][nx_] - dgc));
        }
        const int c = gy * g.nx + gx;
        y[c] = swu[ty + 2][tx + 2] * idt - div;
        y[N + c] = swv[ty + 2][tx + 2] * idt + (dcc * gv[q] + cc * sdgv[ty][tx]) * irho;
    }
}

template <typename T>
cudaError_t launch_jvp_tile(const Geom& g, const JacK<T>* kp, Cache<T> cache, const T* w, T* y, cudaStream_t s,
                            const Members& mb) {
    dim3 grid((g.nx + JT_X - 1) / JT_X, (g.ny + JT_Y - 1) / JT_Y, mb.count);
    jvp_tile_kernel<T><<<grid, JT_THREADS, 0, s>>>(g, kp, cache, w, y, mb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- transpose
// JT = J^T in the same stencil-diagonal storage.  The block of JT at row c, slot s
// (column c + o_s) is the transpose of J's block at row r = c + o_s, slot s' with
// o_s' = -o_s (the slot set is symmetric).  Slots that leave a Neumann domain are 0
// in both.  Used by the adjoint: GMRES on J^T with the Schwarz/ILU(0) preconditioner
// factored from J^T's own subdomain blocks, and the products J0^T mu.
template <typename T, int DIM>
__global__ void __launch_bounds__(256) transpose_kernel(Geom g, const T* __restrict__ J, T* __restrict__ JT) {
    const int N = g.N;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    int x, y, z;
    decode_cell<DIM>(g, c, x, y, z);
    const bool per = g.bc == ACAC_BC_PERIODIC;
#pragma unroll
    for (int s = 0; s < nslot<DIM>(); ++s) {
        const int dx = sl_dx<DIM>(s), dy = sl_dy<DIM>(s), dz = sl_dz<DIM>(s);
        const bool inside = per || (x + dx >= 0 && x + dx < g.nx && y + dy >= 0 && y + dy < g.ny &&
                                    z + dz >= 0 && z + dz < g.nz);
        T b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        if (inside) {
            const int r = slot_nb<DIM>(g, x, y, z, s);
            const int s2 = sl_of<DIM>(-dx, -dy, -dz);
            b0 = J[(size_t)(s2 * 4 + 0) * N + r];
            b1 = J[(size_t)(s2 * 4 + 2) * N + r];
            b2 = J[(size_t)(s2 * 4 + 1) * N + r];
            b3 = J[(size_t)(s2 * 4 + 3) * N + r];
        }
        JT[(size_t)(s * 4 + 0) * N + c] = b0;
        JT[(size_t)(s * 4 + 1) * N + c] = b1;
        JT[(size_t)(s * 4 + 2) * N + c] = b2;
        JT[(size_t)(s * 4 + 3) * N + c] = b3;
    }
}

template <typename T>
cudaError_t launch_transpose(const Geom& g, const T* J, T* JT, cudaStream_t s) {
    if (g.dim == 3) transpose_kernel<T, 3><<<grid1(g.N, 256), 256, 0, s>>>(g, J, JT);
    else transpose_kernel<T, 2><<<grid1(g.N, 256), 256, 0, s>>>(g, J, JT);
    return cudaGetLastError();
}

#define INST(T)                                                                                   \
    template cudaError_t launch_assemble<T>(const Geom&, const JacK<T>*, Cache<T>, T*, cudaStream_t, \
                                            const int*, const Members&);                          \
    template cudaError_t launch_spmv<T>(const Geom&, const T*, const T*, T*, cudaStream_t,        \
                                        const Members&);                                          \
    template cudaError_t launch_jvp_g<T>(const Geom&, const JacK<T>*, Cache<T>, const T*, T*,      \
                                         cudaStream_t, const Members&);                           \
    template cudaError_t launch_jvp_f<T>(const Geom&, const JacK<T>*, Cache<T>, const T*, const T*, \
                                         T*, cudaStream_t, const Members&);                         \
    template cudaError_t launch_jvp_tile<T>(const Geom&, const JacK<T>*, Cache<T>, const T*, T*,    \
                                            cudaStream_t, const Members&);                          \
    template cudaError_t launch_transpose<T>(const Geom&, const T*, T*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace acac
