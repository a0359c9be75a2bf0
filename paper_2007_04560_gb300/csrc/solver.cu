// Host side of the acac C ABI: handle and workspace, the inexact Newton iteration
// with line search (Sec. 3.1, Eq. newton), restarted right-preconditioned GMRES
// (Sec. 3.1, Eq. hjacobi), the subdomain tables of the Schwarz preconditioner, and the
// adaptive time step of Sec. 3.2 (Eq. sencondt, with retry on divergence and eta
// doubling).
//
// A handle holds B >= 1 independent problems (ensemble members) of one grid and one box
// decomposition and solves them in lockstep: every kernel launch covers all members
// (a grid dimension indexes the member), and per-member masks on the device say which
// members take part (those still iterating in Newton, in the line search, in the GMRES
// cycle).  The Givens rotations, the convergence test and the back substitution of
// GMRES run on the device, so a restart cycle is launched without a host read-back per
// Arnoldi step.  A single problem is the case B = 1.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "acac_internal.cuh"

using namespace acac;

// One captured GMRES (Arnoldi) iteration: the graph and, per kernel node, the
// launch accounting (per member taking part) and, when profiling, the event pair
// recorded around it.
struct GraphRec {
    int id;
    double bytes, flops;
    cudaEvent_t a, b;
};
struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<GraphRec> recs;
};

// Per-member device scalars (stride RS doubles): the two Gram-Schmidt passes' Hessenberg
// columns, ||w||^2, the GMRES combination y, the mass-correction shift, and a few slots
// for other reductions (their results land at offset 0).
constexpr int RS_H0 = 0;
constexpr int RS_H1 = MAX_RESTART + 1;
constexpr int RS_NRM = 2 * (MAX_RESTART + 1);
constexpr int RS_Y = 3 * (MAX_RESTART + 1);
constexpr int RS_SHIFT = 4 * (MAX_RESTART + 1);
constexpr int RS = 4 * (MAX_RESTART + 1) + 8;
static_assert(sizeof(GmresHead) == 5 * sizeof(double), "GmresHead holds 5 doubles");

// Masks (B ints each on the device): the members a launch covers.
enum { MK_NEWTON = 0, MK_LS, MK_CYC, MK_GON, MK_RESTART, MK_AUX, MK_COUNT };

struct acac_handle {
    acac_params p;
    Geom g;
    Coef k;                     // member 0's coefficients (the by-value scalars of single-problem calls)
    int B = 1;                  // members
    Members mb;                 // member strides and per-member scalars (mb.on set per launch)
    cudaStream_t stream;        // private stream of all the handle's work
    cudaStream_t user_stream;   // the caller's stream (ordered with `stream` at entry and exit)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    void* jk_dev = nullptr;     // JacK<T> per member of the current linearisation
    MemberK* mk_dev = nullptr;  // per-member coefficients, dt, line-search step
    std::vector<MemberK> mk;    // host copy
    int* masks = nullptr;       // MK_COUNT x B
    std::vector<int> mask_host[MK_COUNT];
    int mask_count[MK_COUNT] = {0};
    int nact = 1;               // members taking part in the launch being issued
    int ncyc = 1;               // members in the current GMRES cycle
    GmresHead* ghead_dev = nullptr;
    GmresWork* gwork_dev = nullptr;
    int* kcnt_dev = nullptr;    // Arnoldi steps of each member's last cycle
    std::vector<GmresHead> ghead;
    int gm_hint = 0;            // steps the previous GMRES cycle took (where to look first)
    // CUDA graphs of the Arnoldi iterations (index j), captured on first use
    std::vector<IterGraph> graphs;
    unsigned graphs_prof = 0;   // timing mask the graphs were captured with
    std::vector<GraphRec>* capture = nullptr;   // non-null while capturing
    int gmres_calls = 0;
    bool mixed;
    size_t N;
    size_t ksz;                 // sizeof Krylov element
    // FP64 state (B members at stride mb.vs)
    double *X, *X0, *Xprev, *Xt, *F, *S, *G, *b, *r, *tmpd, *stage;
    double* lap0 = nullptr;     // Laplacians of X0 during a Newton solve (pass A reads them)
    bool factor_check = false;     // a deferred factorization's flags are still to be read
    bool cache_fresh = false;      // the last residual evaluation wrote the linearisation cache
    // Krylov precision buffers
    void *V, *w, *kt, *jtmp, *cache, *J, *coef, *gscratch;
    void* Zb = nullptr;         // preconditioned basis z_j = M^-1 v_j, restart x ldV (the
                                // solution update is Z y: no preconditioner apply per solve)
    size_t ldV;                 // Krylov basis stride: B members x mb.vs
    // reductions
    double* partial;            // per member: (MAX_RESTART + 3) quantities x blocks
    double* red;                // device results, RS per member
    double* host;               // pinned host mirror of per-member results
    int* flags;                 // [0, B): per-member flags; [B, 2B): sticky apply timeouts
    int* host_flags;            // pinned, 2B
    unsigned* counter;          // reduction counters, one per member (zero between launches)
    // per-member results of the last residual evaluation
    std::vector<double> fn;
    std::vector<int> fl;
    // Schwarz tables
    std::vector<SubInfo> subs;
    std::vector<int> lev;
    std::vector<int> cells3, pos3;   // 3D: level-ordered packed cells, position map
    SubInfo* subs_dev;
    int* lev_dev;
    std::vector<int> rec_of;     // for every grid cell, its records in the boxes (4 per cell in 2D, 8 in
                                 // 3D; -1 unused)
    int* rec_of_dev = nullptr;
    std::vector<unsigned char> own_of;   // 2D: for every grid cell, the slot of rec_of whose box owns it
    unsigned char* own_of_dev = nullptr;
    void* rg = nullptr;          // windowed apply: the right-hand side gathered per box cell, by record
    void* Jp = nullptr;          // Jacobian rows per box cell (52 values each in 2D, 100 in 3D)
    bool jpacked = false;        // Jp holds the current Jacobian (assembled straight into it)
    int *cells3_dev, *pos3_dev;
    // subdomain solves with fill (params.subdomain_solver != ILU(0)): patterns per box shape
    std::vector<SparseShape> sshape;
    SparseShapeDev* sshape_dev = nullptr;
    SparseBox* sbox_dev = nullptr;
    int* sint_dev = nullptr;     // every shape's integer tables
    void* sval = nullptr;        // 2x2 blocks of every box matrix (factored in place)
    void* sdinv = nullptr;       // inverse pivot blocks, 4 values per box cell
    void* sy = nullptr;          // box vectors of the apply when they do not fit shared memory
    int* srec_of_dev = nullptr;  // fill solvers: the box cells (natural order) of every grid cell
    void* zb = nullptr;          // additive extensions (AS, right-RAS): box-cell results by record
    long long sblocks = 0, scells = 0;
    int s_threads = 32, s_fthreads = 512, s_use_map = 1;
    size_t s_fsmem = 0, s_asmem = 0;
    int ras_threads;
    size_t ras_smem;
    RasLaunch ras_launch;
    long long coef_count;
    double nbox;                // cells of all subdomain boxes (overlap counted)
    int ras_maxlev, ras_maxcnt;
    size_t ras_maxpad;
    // time stepping, per member
    std::vector<double> t, dt_prev, eta;
    std::vector<int> nstep;
    std::vector<char> have_prev;
    // kernel launch counts and (when enabled) CUDA-event timings per kernel
    bool prof_on;
    unsigned prof_mask = 0;     // kernel classes timed with events (bit = ACAC_K_*)
    long long launches[ACAC_NKERNEL];
    double kernel_ms[ACAC_NKERNEL];
    double kernel_bytes[ACAC_NKERNEL];   // algorithmic HBM bytes of the counted launches
    double kernel_flops[ACAC_NKERNEL];   // algorithmic floating-point operations
    struct Pending { int id; cudaEvent_t a, b; bool owned_by_graph; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    // adjoint workspace (allocated on first use): mu, lam, lam2, target (2N doubles each)
    // and one stencil matrix in the Krylov precision
    double* adj = nullptr;
    void* adjJ = nullptr;
};

namespace {

struct Err {
    int code;
};

#define CU(call)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) throw Err{e_ == cudaErrorMemoryAllocation ? ACAC_E_NOMEM : ACAC_E_CUDA}; \
    } while (0)

template <typename P>
void dmalloc(P** ptr, size_t bytes) {
    void* q = nullptr;
    CU(cudaMalloc(&q, bytes ? bytes : 16));
    *ptr = (P*)q;
}

cudaEvent_t take_event(acac_handle* h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    return e;
}

// Adds the durations of completed timed launches (call after a stream sync).
void prof_collect(acac_handle* h) {
    for (auto& p : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) h->kernel_ms[p.id] += ms;
        if (p.owned_by_graph) continue;
        h->pool.push_back(p.a);
        h->pool.push_back(p.b);
    }
    h->pending.clear();
}

// Brackets one kernel launch: counts it (bytes and flops per member taking part) and,
// when profiling, records CUDA events around it on the handle's stream.
struct KScope {
    acac_handle* h;
    cudaEvent_t b;
    KScope(acac_handle* h_, int id, double bytes = 0.0, double flops = 0.0) : h(h_), b(nullptr) {
        if (h->capture) {
            // inside a graph capture: the accounting happens at every replay (scaled by the
            // members of the cycle then), and the events (when profiling) become
            // event-record nodes of the graph
            GraphRec r{id, bytes, flops, nullptr, nullptr};
            if (h->prof_on && (h->prof_mask >> id & 1u)) {
                // events come from the pool, stocked before the capture began
                if (h->pool.size() < 2) throw Err{ACAC_E_CUDA};
                r.a = h->pool.back();
                h->pool.pop_back();
                r.b = h->pool.back();
                h->pool.pop_back();
                CU(cudaEventRecordWithFlags(r.a, h->stream, cudaEventRecordExternal));
                b = r.b;
            }
            h->capture->push_back(r);
            return;
        }
        h->launches[id]++;
        h->kernel_bytes[id] += bytes * h->nact;
        h->kernel_flops[id] += flops * h->nact;
        if (h->prof_on && (h->prof_mask >> id & 1u)) {
            cudaEvent_t a = take_event(h);
            b = take_event(h);
            CU(cudaEventRecord(a, h->stream));
            h->pending.push_back({id, a, b, false});
        }
    }
    ~KScope() {
        if (!b) return;
        if (h->capture) cudaEventRecordWithFlags(b, h->stream, cudaEventRecordExternal);
        else cudaEventRecord(b, h->stream);
    }
};

// Orders the handle's private stream after the caller's stream on entry to a C-ABI
// call and the caller's stream after the private stream on exit.
struct Join {
    acac_handle* h;
    explicit Join(acac_handle* h_) : h(h_) {
        if (!h->ev_in) return;
        cudaEventRecord(h->ev_in, h->user_stream);
        cudaStreamWaitEvent(h->stream, h->ev_in, 0);
    }
    ~Join() {
        if (!h->ev_in) return;
        cudaEventRecord(h->ev_out, h->stream);
        cudaStreamWaitEvent(h->user_stream, h->ev_out, 0);
    }
};

void free_graphs(acac_handle* h) {
    for (auto& G : h->graphs) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        for (auto& r : G.recs) {
            if (r.a) cudaEventDestroy(r.a);
            if (r.b) cudaEventDestroy(r.b);
        }
    }
    h->graphs.clear();
}

#define KL(id, call)                 \
    do {                             \
        KScope ks_(h, id);           \
        CU(call);                    \
    } while (0)
// Same, with the launch's algorithmic HBM bytes and floating-point operations per member.
#define KLA(id, bytes, flops, call)          \
    do {                                     \
        KScope ks_(h, id, (bytes), (flops)); \
        CU(call);                            \
    } while (0)

// Member 0's cache fields; member m's are at m * mb.cs (member_cache).
template <typename T>
Cache<T> cache_of(acac_handle* h) {
    T* base = (T*)h->cache;
    const size_t N = h->N;
    return Cache<T>{base, base + N, base + 2 * N, base + 3 * N, base + 4 * N, base + 5 * N, base + 6 * N};
}

// Reduction target: partials, member results at out (+ m * RS), counters.
Red red_to(acac_handle* h, double* out) { return Red{h->partial, out, h->counter}; }

// ---------------------------------------------------------------- members
// Every member takes part (single-problem calls, whole-ensemble work).
Members all_members(acac_handle* h) {
    h->nact = h->B;
    return h->mb;
}

// The members of mask `slot`.
Members on_mask(acac_handle* h, int slot) {
    Members mb = h->mb;
    mb.on = h->masks + (size_t)slot * h->B;
    h->nact = slot == MK_GON ? h->ncyc : h->mask_count[slot];
    return mb;
}

// Writes mask `slot` (when it changed: the copy from pageable memory is staged at once, so
// the host vector may change right after).
void set_mask(acac_handle* h, int slot, const std::vector<int>& v) {
    int cnt = 0;
    for (int x : v) cnt += x ? 1 : 0;
    h->mask_count[slot] = cnt;
    if (h->mask_host[slot] == v) return;
    h->mask_host[slot] = v;
    CU(cudaMemcpyAsync(h->masks + (size_t)slot * h->B, h->mask_host[slot].data(), sizeof(int) * h->B,
                       cudaMemcpyHostToDevice, h->stream));
}

int any_of(const std::vector<int>& v) {
    for (int x : v)
        if (x) return 1;
    return 0;
}

// Per-member scalars to the device: coefficients, dt and line-search step, and the
// Jacobian scalars formed from them.
template <typename T>
void write_members(acac_handle* h) {
    CU(cudaMemcpyAsync(h->mk_dev, h->mk.data(), sizeof(MemberK) * h->B, cudaMemcpyHostToDevice, h->stream));
    std::vector<JacK<T>> jk(h->B);
    for (int m = 0; m < h->B; ++m) {
        const MemberK& q = h->mk[m];
        jk[m] = jac_consts<T>(Coef{q.alpha, q.beta, q.theta, q.gamma, q.rho, h->p.taylor_S}, q.dt);
    }
    CU(cudaMemcpyAsync(h->jk_dev, jk.data(), sizeof(JacK<T>) * h->B, cudaMemcpyHostToDevice, h->stream));
}
void write_members_any(acac_handle* h) {
    if (h->mixed) write_members<float>(h);
    else write_members<double>(h);
}
// A single problem's dt (member 0), for the component entry points.
void set_dt0(acac_handle* h, double dt) {
    for (auto& q : h->mk) q.dt = dt;
    write_members_any(h);
}

// n scalars of every member from red + off into host[m * n + i]; synchronises.
void read_member_scalars(acac_handle* h, size_t off, int n) {
    CU(cudaMemcpy2DAsync(h->host, sizeof(double) * n, h->red + off, sizeof(double) * RS, sizeof(double) * n,
                         h->B, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    prof_collect(h);
}

// Member 0's first scalars (single-problem helpers).
double read_scalars(acac_handle* h, int n) {
    CU(cudaMemcpyAsync(h->host, h->red, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    prof_collect(h);
    return h->host[0];
}

// Per-member flags (both halves) to host_flags; the caller synchronises.
void fetch_flags(acac_handle* h) {
    CU(cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int) * 2 * h->B, cudaMemcpyDeviceToHost, h->stream));
}

// F at the members of mask `slot` (slot < 0: every member): at X, or (trial) at the
// line-search state X + lam (S + shift e_u) with lam and the shift per member on the
// device.  With fill_cache pass A also writes the linearisation cache at the evaluated
// state, which the next Newton iteration uses if the line search accepts that state.
// Sets h->fn[m] = ||F|| and h->fl[m] (bit 0: a midpoint left the admissible set, bit 1:
// the trial state did, bit 3: a Schwarz apply gave up a bounded wait, sticky) for the
// members of the mask.
void eval_residual(acac_handle* h, int slot, const double* X, bool trial, bool use_lap0 = false,
                   bool fill_cache = false) {
    const Members mb = slot < 0 ? all_members(h) : on_mask(h, slot);
    CU(cudaMemsetAsync(h->flags, 0, sizeof(int) * h->B, h->stream));
    ResidualArgs a;
    if (fill_cache && use_lap0) {
        if (h->mixed) {
            a.cache_mode = 2;
            a.cache_f = cache_of<float>(h);
        } else {
            a.cache_mode = 1;
            a.cache_d = cache_of<double>(h);
        }
    }
    h->cache_fresh = a.cache_mode != 0;
    a.X = X; a.S = trial ? h->S : nullptr; a.lam = 0.0; a.shift = 0.0; a.X0 = h->X0; a.dt = h->mk[0].dt;
    a.L0 = use_lap0 ? h->lap0 : nullptr;
    a.same = use_lap0 && !trial && X == h->X0;
    a.shift_sum = trial ? h->red + RS_SHIFT : nullptr;
    a.shift_scale = 1.0 / (double)h->N;
    a.Xt = h->Xt; a.G = h->G; a.F = h->F; a.red = red_to(h, h->red); a.flags = h->flags;
    if (trial) {
        KLA(ACAC_K_VECTOR, 40.0 * h->N, 0.0, launch_trial(h->g, a, h->stream, mb));
        a.X = h->Xt;
        a.S = nullptr;
    }
    // pass A: ~113 FP64 operations per cell in the formulas (midpoints, Laplacians of the new
    // state, series arguments with one reciprocal, two table logarithms, four series of K = 4
    // terms, G and the mobility), charged as 2 flop-equivalents each (one DFMA slot).  At the
    // start state (a.same) the differences, the series and their arguments and the Laplacian
    // of X drop out: ~57 operations, and X is not read apart from X0
    KLA(ACAC_K_RESIDUAL_G, 8.0 * h->N * (a.same ? 5 : 7) + (a.cache_mode ? 7.0 * h->ksz * h->N : 0.0),
        (a.same ? 114.0 : 226.0) * h->N, launch_residual_g(h->g, h->k, a, h->stream, mb));
    KLA(ACAC_K_RESIDUAL_F, 8.0 * h->N * 9, 30.0 * h->N, launch_residual_f(h->g, h->k, a, h->stream, mb));
    fetch_flags(h);
    read_member_scalars(h, 0, 1);
    for (int m = 0; m < h->B; ++m) {
        h->fn[m] = sqrt(h->host[m]);
        h->fl[m] = h->host_flags[m] | (h->host_flags[h->B + m] ? 8 : 0);
    }
}

template <typename T>
void jvp_action(acac_handle* h, const Members& mb, const T* w, T* y) {
    const JacK<T>* kp = (const JacK<T>*)h->jk_dev;
    if (h->g.dim == 2 && sizeof(T) == 4) {
        // FP32: one tiled pass (HBM bound); FP64 keeps the two passes (FP64-pipe bound,
        // no halo recomputation)
        KLA(ACAC_K_JVP_F, (double)sizeof(T) * h->N * 11, 80.0 * h->N,
            launch_jvp_tile<T>(h->g, kp, cache_of<T>(h), w, y, h->stream, mb));
        return;
    }
    KLA(ACAC_K_JVP_G, (double)sizeof(T) * h->N * 9, 32.0 * h->N,
        launch_jvp_g<T>(h->g, kp, cache_of<T>(h), w, (T*)h->jtmp, h->stream, mb));
    KLA(ACAC_K_JVP_F, (double)sizeof(T) * h->N * 10, 48.0 * h->N,
        launch_jvp_f<T>(h->g, kp, cache_of<T>(h), w, (const T*)h->jtmp, y, h->stream, mb));
}

template <typename T>
void jac_action(acac_handle* h, const Members& mb, const T* w, T* y) {
    if (h->p.jac_mode == ACAC_JAC_ASSEMBLED)
        KLA(ACAC_K_SPMV, (double)sizeof(T) * h->N * 56, 104.0 * h->N,
            launch_spmv<T>(h->g, (const T*)h->J, w, y, h->stream, mb));
    else
        jvp_action<T>(h, mb, w, y);
}

template <typename T>
void precond(acac_handle* h, const Members& mb, const T* r, T* z) {
    int* err = h->flags + h->B;   // sticky timeout flags
    if (h->p.subdomain_solver != ACAC_SUB_ILU0) {
        KLA(ACAC_K_RAS_APPLY, (double)sizeof(T) * (4.0 * h->sblocks + 4.0 * h->scells + 4.0 * h->N),
            16.0 * h->sblocks,
            launch_sparse_apply<T>(h->g, (int)h->subs.size(), h->subs_dev, h->sbox_dev, h->sshape_dev,
                                   (const T*)h->sval, (const T*)h->sdinv, r, z, h->p.ras_type, (T*)h->sy,
                                   h->s_threads, h->s_asmem, h->stream, mb, h->srec_of_dev, (T*)h->zb));
        return;
    }
    if (h->g.dim == 3) {
        KLA(ACAC_K_RAS_APPLY, (double)sizeof(T) * (104.0 * h->nbox + 4.0 * h->N), 200.0 * h->nbox,
            launch_ras_apply3<T>(h->g, (int)h->subs.size(), h->subs_dev, h->lev_dev, h->cells3_dev,
                                 (const T*)h->coef, r, z, h->p.ras_type, h->ras_launch, (T*)h->gscratch,
                                 err, h->stream, mb, h->rec_of_dev, (T*)h->zb));
        return;
    }
    if (h->ras_launch.window && sizeof(T) == 4)
        KLA(ACAC_K_VECTOR, (double)sizeof(T) * (2.0 * h->N + 2.0 * h->nbox) + 17.0 * h->N, 0.0,
            launch_ras_gather<T>(h->g, r, h->rec_of_dev, h->own_of_dev, h->p.ras_type, (T*)h->rg, h->stream, mb));
    KLA(ACAC_K_RAS_APPLY, (double)sizeof(T) * (54.0 * h->nbox + 2.0 * h->N), 104.0 * h->nbox,
        launch_ras_apply<T>(h->g, (int)h->subs.size(), h->subs_dev, h->lev_dev, (const T*)h->coef, r, z,
                            h->p.ras_type, h->ras_launch.threads, h->ras_launch, (T*)h->gscratch,
                            sizeof(T) == 4 ? (const T*)h->rg : nullptr, err, h->stream, mb, h->rec_of_dev,
                            (T*)h->zb));
}

// Subdomain factorizations of the members in mb.  With defer, the pivot / timeout flags
// are read with the next GMRES read-back (one host round trip fewer per Newton step) and
// ACAC_OK is returned; without, member 0's status.
template <typename T>
int factor(acac_handle* h, const Members& mb, bool defer = false) {
    CU(cudaMemsetAsync(h->flags, 0, sizeof(int) * h->B, h->stream));
    auto done = [&](bool timeout_bit) -> int {
        if (defer) {
            h->factor_check = true;
            return ACAC_OK;
        }
        fetch_flags(h);
        CU(cudaStreamSynchronize(h->stream));
        prof_collect(h);
        const int f = h->host_flags[0];
        return (timeout_bit && (f & 8)) ? ACAC_E_TIMEOUT : f ? ACAC_E_DIVERGED : ACAC_OK;
    };
    if (h->p.subdomain_solver != ACAC_SUB_ILU0) {
        // A_k of every box from the stencil-diagonal Jacobian, then the block IKJ
        // elimination on the ILU(1) / ILU(2) / LU pattern
        CU(cudaMemsetAsync(h->sval, 0, (size_t)h->mb.cfs * h->B * sizeof(T), h->stream));
        KLA(ACAC_K_REPACK, (double)sizeof(T) * (4.0 * h->sblocks + 4.0 * (h->g.dim == 3 ? NSLOT3 : NSLOT) * h->N),
            0.0,
            launch_sparse_init<T>(h->g, (int)h->subs.size(), h->subs_dev, h->sbox_dev, h->sshape_dev,
                                  (const T*)h->J, (T*)h->sval, h->stream, mb));
        KLA(ACAC_K_RAS_FACTOR, (double)sizeof(T) * 8.0 * h->sblocks, 0.0,
            launch_sparse_factor<T>((int)h->subs.size(), h->sbox_dev, h->sshape_dev, (T*)h->sval, (T*)h->sdinv,
                                    h->flags, h->s_fthreads, h->s_fsmem, h->s_use_map, h->stream, mb));
        return done(true);
    }
    if (h->g.dim == 3) {
        int packed3 = h->jpacked ? 1 : 0;
        if (!packed3 && sizeof(T) == 4) {
            KLA(ACAC_K_REPACK, (double)sizeof(T) * (100.0 * h->N + 100.0 * h->nbox), 0.0,
                launch_repack<T>(h->g, (const T*)h->J, h->rec_of_dev, (T*)h->Jp, h->stream, mb));
            packed3 = 1;
        }
        KLA(ACAC_K_RAS_FACTOR, (double)sizeof(T) * 200.0 * h->nbox, 1200.0 * h->nbox,
            launch_ras_factor3<T>(h->g, (int)h->subs.size(), h->subs_dev, h->lev_dev, h->cells3_dev, h->pos3_dev,
                                  packed3 ? (const T*)h->Jp : (const T*)h->J, packed3, (T*)h->coef,
                                  h->ras_threads, h->flags, h->stream, mb));
        return done(false);
    }
    const int ring_cells = h->ras_maxcnt;
    const size_t smem = sizeof(int) * (size_t)(((h->ras_maxlev + 1 + 3) & ~3) + 3 & ~3) +
                        sizeof(T) * 5 * (size_t)ring_cells * CREC;
    // the factorization reads each cell's rows: from the per-box records when the assembly
    // wrote them; else repacked first in FP32 (the stencil-diagonal reads waste DRAM
    // sectors), directly in FP64 (bound by the FP64 pipe, where the repack does not pay)
    int packed = h->jpacked ? 1 : 0;
    if (!packed && sizeof(T) == 4) {
        KLA(ACAC_K_REPACK, (double)sizeof(T) * (52.0 * h->N + 52.0 * h->nbox), 0.0,
            launch_repack<T>(h->g, (const T*)h->J, h->rec_of_dev, (T*)h->Jp, h->stream, mb));
        packed = 1;
    }
    KLA(ACAC_K_RAS_FACTOR, (double)sizeof(T) * 104.0 * h->nbox, 528.0 * h->nbox,
        launch_ras_factor<T>(h->g, (int)h->subs.size(), h->subs_dev, h->lev_dev,
                             packed ? (const T*)h->Jp : (const T*)h->J, packed, (T*)h->coef,
                             h->ras_threads, ring_cells, smem, h->flags, h->stream, mb));
    return done(false);
}

// One Arnoldi step of GMRES for the members still iterating (mask MK_GON): v_{j+1} =
// J M^{-1} v_j orthogonalised against v_0..v_j by classical Gram–Schmidt (twice when
// cgs_refine) and normalised, then the member's Givens step on the device (which clears
// its MK_GON entry once it has converged or stopped).
template <typename T>
void arnoldi_step(acac_handle* h, int j) {
    const long long n = 2 * (long long)h->N;
    const Members mb = on_mask(h, MK_GON);
    T* V = (T*)h->V;
    const long long ld = (long long)h->ldV;
    T* vj = V + (size_t)j * ld;
    T* vn = V + (size_t)(j + 1) * ld;
    T* zj = (T*)h->Zb + (size_t)j * ld;
    precond<T>(h, mb, vj, zj);
    jac_action<T>(h, mb, (const T*)zj, vn);
    const int passes = h->p.cgs_refine ? 2 : 1;
    for (int pass = 0; pass < passes; ++pass) {
        double* hcol = h->red + (pass ? RS_H1 : RS_H0);
        KLA(ACAC_K_DOT, (double)sizeof(T) * n * (j + 2), 2.0 * n * (j + 1),
            launch_multi_dot<T>(V, ld, j + 1, vn, n, red_to(h, hcol), h->stream, mb));
        const bool last = pass == passes - 1;
        KLA(ACAC_K_CGS_UPDATE, (double)sizeof(T) * n * (j + 3), 2.0 * n * (j + 2),
            launch_cgs_update<T>(V, ld, j + 1, hcol, vn, n, last ? 1 : 0, red_to(h, h->red + RS_NRM), h->stream,
                                 mb));
    }
    KL(ACAC_K_VECTOR, launch_scale_from<T>(vn, h->red + RS_NRM, vn, n, h->stream, mb));
    KL(ACAC_K_VECTOR, launch_gmres_givens(h->ghead_dev, h->gwork_dev, h->red, RS, j, passes,
                                          h->masks + (size_t)MK_GON * h->B, h->B, h->stream));
}

// arnoldi_step(j), replayed from a CUDA graph captured on its first use (one graph per
// j; every pointer the step's kernels take is fixed for the handle's lifetime and their
// scalars live on the device), or launched directly.  Does not synchronise.
template <typename T>
void arnoldi_launch(acac_handle* h, int j) {
    const bool use_graph = h->p.graphs && h->gmres_calls > 0;
    if (!use_graph) {
        arnoldi_step<T>(h, j);
        return;
    }
    const unsigned timing = h->prof_on ? h->prof_mask : 0u;
    if (h->graphs_prof != timing) {
        free_graphs(h);
        h->graphs_prof = timing;
    }
    if ((int)h->graphs.size() <= j) h->graphs.resize(j + 1);
    IterGraph& G = h->graphs[j];
    if (!G.exec) {
        if (h->prof_on)
            while (h->pool.size() < 32) {
                cudaEvent_t e;
                CU(cudaEventCreate(&e));
                h->pool.push_back(e);
            }
        cudaGraph_t graph = nullptr;
        CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        h->capture = &G.recs;
        try {
            arnoldi_step<T>(h, j);
        } catch (Err e) {
            h->capture = nullptr;
            cudaStreamEndCapture(h->stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        h->capture = nullptr;
        CU(cudaStreamEndCapture(h->stream, &graph));
        const cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        CU(e);
    }
    CU(cudaGraphLaunch(G.exec, h->stream));
    for (const GraphRec& r : G.recs) {
        h->launches[r.id]++;
        // counted for every member of the cycle (those that have already converged
        // return at once)
        h->kernel_bytes[r.id] += r.bytes * h->ncyc;
        h->kernel_flops[r.id] += r.flops * h->ncyc;
        if (r.a) h->pending.push_back({r.id, r.a, r.b, true});
    }
}

// Restarted GMRES for J x = b, b = bsign * bsrc (bsrc = h->b when null; bsign = +-1, an
// exact sign: the Newton loop's b = -F is read from F itself), x0 = 0, right
// preconditioning, for the members in `want`.  x (device, member stride mb.vs) receives the
// solutions; per member gst (ACAC_OK, ACAC_E_DIVERGED or ACAC_E_TIMEOUT), gits (iterations)
// and gres (residual estimate).  bnorm: ||b|| per member when already known (the Newton
// loop's b = -F has the norm of its residual evaluation; no reduction and read-back are
// spent on it), else null.  With defer_timeout the apply's sticky timeout flags are left to
// the caller's next read-back.
template <typename T>
void gmres(acac_handle* h, const std::vector<int>& want, double* x, std::vector<int>& gst, std::vector<int>& gits,
           std::vector<double>& gres, const std::vector<double>* bnorm, bool defer_timeout = false,
           const double* bsrc = nullptr, double bsign = 1.0) {
    if (!bsrc) bsrc = h->b;
    // the first call runs eagerly (it also sets the kernels' shared-memory limits); later
    // calls replay captured graphs
    struct Count {
        acac_handle* h;
        ~Count() { h->gmres_calls++; }
    } count{h};
    const int B = h->B;
    const long long n = 2 * (long long)h->N;
    const int mres = h->p.gmres_restart;
    const long long ld = (long long)h->ldV;
    T* tt = (T*)h->kt;
    T* w = (T*)h->w;
    int* gon_host = h->host_flags + 2 * B;
    gst.assign(B, ACAC_OK);
    gits.assign(B, 0);
    gres.assign(B, 0.0);
    CU(cudaMemsetAsync(x, 0, sizeof(double) * h->mb.vs * B, h->stream));
    // a deferred factorization's flags come back with the first read-back of the solve
    bool flags_pending = h->factor_check;
    h->factor_check = false;
    auto factor_flags = [&]() {   // after a synchronised fetch_flags
        if (!flags_pending) return;
        flags_pending = false;
        for (int m = 0; m < B; ++m) {
            if (!want[m]) continue;
            const int f = h->host_flags[m];
            if (f & 8) gst[m] = ACAC_E_TIMEOUT;
            else if (f) gst[m] = ACAC_E_DIVERGED;
        }
    };
    std::vector<double> beta(B, 0.0), tol(B, 0.0);
    if (bnorm) {
        beta = *bnorm;
    } else {
        set_mask(h, MK_AUX, want);
        KL(ACAC_K_VECTOR, launch_norm2_double(bsrc, nullptr, n, red_to(h, h->red), h->stream, on_mask(h, MK_AUX)));
        if (flags_pending) fetch_flags(h);
        read_member_scalars(h, 0, 1);
        for (int m = 0; m < B; ++m) beta[m] = sqrt(h->host[m]);
        factor_flags();
    }
    std::vector<int> act(B, 0);
    for (int m = 0; m < B; ++m) {
        if (!want[m]) continue;
        tol[m] = std::max(h->p.gmres_rtol * beta[m], h->p.gmres_atol);
        gres[m] = beta[m];
        act[m] = gst[m] == ACAC_OK && beta[m] > tol[m];
    }
    const double* rsrc = bsrc;
    double rsign = bsign;
    h->ghead.resize(B);
    while (any_of(act)) {
        // cycle start: v_0 = r / beta, g = beta e_1
        for (int m = 0; m < B; ++m)
            h->ghead[m] = GmresHead{beta[m], tol[m], beta[m], gits[m], h->p.gmres_maxit, 0, GMRES_RUNNING};
        CU(cudaMemcpyAsync(h->ghead_dev, h->ghead.data(), sizeof(GmresHead) * B, cudaMemcpyHostToDevice, h->stream));
        set_mask(h, MK_CYC, act);
        h->ncyc = h->mask_count[MK_CYC];
        int* cyc = h->masks + (size_t)MK_CYC * B;
        KL(ACAC_K_VECTOR, launch_gmres_start(h->ghead_dev, h->gwork_dev, cyc, h->masks + (size_t)MK_GON * B, B,
                                             h->stream));
        KL(ACAC_K_VECTOR, launch_to_krylov<T>(rsrc, rsign, (T*)h->V, n, h->stream, on_mask(h, MK_CYC),
                                              (const double*)h->ghead_dev, (int)(sizeof(GmresHead) / sizeof(double))));
        // Arnoldi steps without read-backs: the first look at the members' progress comes
        // after as many steps as the previous cycle took, then one after every step
        int j = 0;
        int next = std::max(1, std::min(mres, h->gm_hint));
        while (j < mres) {
            arnoldi_launch<T>(h, j);
            ++j;
            if (j >= mres || j < next) continue;
            if (flags_pending) fetch_flags(h);
            CU(cudaMemcpyAsync(gon_host, h->masks + (size_t)MK_GON * B, sizeof(int) * B, cudaMemcpyDeviceToHost,
                               h->stream));
            CU(cudaStreamSynchronize(h->stream));
            prof_collect(h);
            factor_flags();
            bool any = false;
            for (int m = 0; m < B; ++m) any = any || gon_host[m];
            if (!any) break;
            next = j + 1;
        }
        // y = R^-1 g and x += Z y (z_j = M^-1 v_j kept by the Arnoldi steps: the
        // preconditioner is linear) for the members of the cycle
        KL(ACAC_K_VECTOR, launch_gmres_solve(h->ghead_dev, h->gwork_dev, cyc, h->red + RS_Y, RS, h->kcnt_dev, B,
                                             h->stream));
        const Members mc = on_mask(h, MK_CYC);
        KL(ACAC_K_VECTOR, launch_lincomb<T>((const T*)h->Zb, ld, mres, h->red + RS_Y, tt, n, h->stream, mc,
                                            h->kcnt_dev));
        KL(ACAC_K_VECTOR, launch_axpy_to_double<T>(1.0, tt, x, n, h->stream, mc));
        CU(cudaMemcpyAsync(h->ghead.data(), h->ghead_dev, sizeof(GmresHead) * B, cudaMemcpyDeviceToHost, h->stream));
        if (flags_pending) fetch_flags(h);
        CU(cudaStreamSynchronize(h->stream));
        prof_collect(h);
        factor_flags();
        int hint = 0;
        std::vector<int> rst(B, 0);
        for (int m = 0; m < B; ++m) {
            if (!act[m]) continue;
            const GmresHead& H = h->ghead[m];
            gits[m] = H.its;
            gres[m] = H.resid;
            hint = std::max(hint, H.k);
            act[m] = 0;
            if (gst[m] != ACAC_OK) continue;
            if (H.status == GMRES_LIMIT || H.status == GMRES_NONFINITE) gst[m] = ACAC_E_DIVERGED;
            else if (H.status == GMRES_RUNNING) rst[m] = 1;
        }
        h->gm_hint = hint;
        if (!any_of(rst)) break;
        // restart: r = b - J x
        set_mask(h, MK_RESTART, rst);
        const Members mr = on_mask(h, MK_RESTART);
        KL(ACAC_K_VECTOR, launch_to_krylov<T>(x, 1.0, tt, n, h->stream, mr));
        jac_action<T>(h, mr, tt, w);
        KL(ACAC_K_VECTOR, launch_residual_restart<T>(bsrc, bsign, w, h->r, n, red_to(h, h->red), h->stream, mr));
        read_member_scalars(h, 0, 1);
        for (int m = 0; m < B; ++m) {
            if (!rst[m]) continue;
            beta[m] = sqrt(h->host[m]);
            if (beta[m] <= tol[m]) gres[m] = beta[m];
            else act[m] = 1;
        }
        rsrc = h->r;
        rsign = 1.0;
    }
    if (flags_pending || !defer_timeout) {
        fetch_flags(h);
        CU(cudaStreamSynchronize(h->stream));
        prof_collect(h);
        factor_flags();
        if (!defer_timeout)
            for (int m = 0; m < B; ++m)
                if (want[m] && gst[m] == ACAC_OK && h->host_flags[B + m]) gst[m] = ACAC_E_TIMEOUT;
    }
}

// fresh: the cache already holds the linearisation at X (written by the residual evaluation
// that produced X, see eval_residual)
template <typename T>
void linearize_and_maybe_assemble(acac_handle* h, const Members& mb, const double* X, bool assemble,
                                  bool fresh = false) {
    if (!fresh) {
        // single problems only: the Newton loop's evaluations always leave the cache fresh
        if (h->B != 1) throw Err{ACAC_E_ARG};
        KLA(ACAC_K_LINEARIZE, 56.0 * h->N + 7.0 * sizeof(T) * h->N, 0.0,
            launch_linearize<T>(h->g, h->k, X, h->X0, h->G, cache_of<T>(h), h->stream));
    }
    h->cache_fresh = false;
    if (!assemble) return;
    const JacK<T>* kp = (const JacK<T>*)h->jk_dev;
    // with matrix-free products the assembled Jacobian feeds only the subdomain
    // factorization: in 2D assemble it straight into the factorization's records
    h->jpacked = h->p.jac_mode == ACAC_JAC_MATFREE && h->p.subdomain_solver == ACAC_SUB_ILU0;
    if (h->jpacked)
        KLA(ACAC_K_ASSEMBLE, (double)sizeof(T) * (7.0 * h->N + 4.0 * (h->g.dim == 3 ? NSLOT3 : NSLOT) * h->nbox), 0.0,
            launch_assemble<T>(h->g, kp, cache_of<T>(h), (T*)h->Jp, h->stream, h->rec_of_dev, mb));
    else
        KLA(ACAC_K_ASSEMBLE, (double)sizeof(T) * 59.0 * h->N, 0.0,
            launch_assemble<T>(h->g, kp, cache_of<T>(h), (T*)h->J, h->stream, nullptr, mb));
}

// The line-search steps (and the rest of the per-member scalars) to the device.
void write_lam(acac_handle* h) {
    CU(cudaMemcpyAsync(h->mk_dev, h->mk.data(), sizeof(MemberK) * h->B, cudaMemcpyHostToDevice, h->stream));
}

// Newton iteration (Sec. 3.1) from X_0 = X0 for the members in `want`, each with its own
// dt (h->mk, already on the device).  Roots in h->X; st[m] per member; info[m] accumulates
// the member's iteration counts.
template <typename T>
void nks(acac_handle* h, const std::vector<int>& want, std::vector<int>& st, acac_step_info* info) {
    const int B = h->B;
    const size_t N = h->N;
    const long long n = 2 * (long long)N;
    st.assign(B, ACAC_OK);
    std::vector<int> act = want;
    std::vector<double> fnorm(B, 0.0), stop(B, 0.0);
    std::vector<const double*> root(B, nullptr);
    set_mask(h, MK_NEWTON, act);
    // X0 stays fixed over the solve: its Laplacians once, for every pass A of the solve
    KLA(ACAC_K_VECTOR, 32.0 * N, 0.0, launch_laplacian(h->g, h->X0, h->lap0, h->stream, on_mask(h, MK_NEWTON)));
    // the current iterate: the start state X0 itself (read in place), then the accepted
    // trial states, which alternate between the buffers X and Xt
    const double* cur = h->X0;
    eval_residual(h, MK_NEWTON, cur, false, true, true);
    for (int m = 0; m < B; ++m) {
        if (!want[m]) continue;
        info[m].fnorm0 = info[m].fnorm = fnorm[m] = h->fn[m];
        if (h->fl[m] & 1) {
            st[m] = ACAC_E_DOMAIN;
            act[m] = 0;
        } else if (!isfinite(fnorm[m])) {
            st[m] = ACAC_E_DIVERGED;
            act[m] = 0;
        } else {
            stop[m] = std::max(h->p.newton_rtol * fnorm[m], h->p.newton_atol);
            if (fnorm[m] <= stop[m]) {
                act[m] = 0;
                root[m] = cur;
            }
        }
    }
    std::vector<int> gst, gits;
    std::vector<double> gres;
    for (int it = 0; any_of(act); ++it) {
        if (it >= h->p.newton_maxit) {
            for (int m = 0; m < B; ++m)
                if (act[m]) st[m] = ACAC_E_DIVERGED;
            break;
        }
        set_mask(h, MK_NEWTON, act);
        const bool refactor = (it == 0) || !h->p.ilu_reuse;
        linearize_and_maybe_assemble<T>(h, on_mask(h, MK_NEWTON), cur,
                                        refactor || h->p.jac_mode == ACAC_JAC_ASSEMBLED, h->cache_fresh);
        if (refactor) {
            factor<T>(h, on_mask(h, MK_NEWTON), true);
            for (int m = 0; m < B; ++m) info[m].ilu_factorizations += act[m];
        }
        // b = -F, read from F with the sign folded into GMRES's first basis vector
        gmres<T>(h, act, h->S, gst, gits, gres, &fnorm, true, h->F, -1.0);
        for (int m = 0; m < B; ++m) {
            if (!act[m]) continue;
            info[m].gmres_its += gits[m];
            if (gst[m] != ACAC_OK) {
                st[m] = gst[m];
                act[m] = 0;
            }
        }
        if (!any_of(act)) break;
        set_mask(h, MK_NEWTON, act);
        // shift S_u by a constant so that sum(u + S_u) = sum(u^n); the sums stay on the
        // device, where the trial kernel reads them
        KL(ACAC_K_VECTOR, launch_sum_pair(h->X0, cur, h->S, (long long)N, red_to(h, h->red + RS_SHIFT), h->stream,
                                          on_mask(h, MK_NEWTON)));
        std::vector<int> ls = act;
        std::vector<double> lam(B, 1.0), ft(B, 0.0);
        while (any_of(ls)) {
            for (int m = 0; m < B; ++m) h->mk[m].lam = lam[m];
            write_lam(h);
            set_mask(h, MK_LS, ls);
            eval_residual(h, MK_LS, cur, true, true, true);
            for (int m = 0; m < B; ++m) {
                if (!ls[m]) continue;
                const double f = h->fn[m];
                if (h->fl[m] & 8) {
                    st[m] = ACAC_E_TIMEOUT;
                    act[m] = ls[m] = 0;
                } else if (h->fl[m] == 0 && isfinite(f) && f * f <= (1.0 - 2e-4 * lam[m]) * fnorm[m] * fnorm[m]) {
                    ft[m] = f;
                    ls[m] = 0;
                } else {
                    lam[m] *= 0.5;
                    info[m].line_search_cuts++;
                    if (lam[m] < 1.0 / 1024.0) {
                        st[m] = ACAC_E_DIVERGED;
                        act[m] = ls[m] = 0;
                    }
                }
            }
        }
        // the accepted states of the members still iterating are in Xt; members that
        // finished earlier keep their roots where they were (root[m])
        std::swap(h->X, h->Xt);
        cur = h->X;
        for (int m = 0; m < B; ++m) {
            if (!act[m]) continue;
            fnorm[m] = ft[m];
            info[m].newton_its = it + 1;
            info[m].fnorm = fnorm[m];
            if (fnorm[m] <= stop[m]) {
                act[m] = 0;
                root[m] = cur;
            }
        }
    }
    // roots elsewhere than X: left in Xt by later swaps, or the start state itself
    for (const double* src : {(const double*)h->Xt, (const double*)h->X0}) {
        std::vector<int> fix(B, 0);
        for (int m = 0; m < B; ++m) fix[m] = want[m] && st[m] == ACAC_OK && root[m] == src;
        if (!any_of(fix)) continue;
        set_mask(h, MK_AUX, fix);
        KLA(ACAC_K_VECTOR, 32.0 * N, 0.0, launch_copy_members(src, h->X, n, h->stream, on_mask(h, MK_AUX)));
    }
}

void nks_dispatch(acac_handle* h, const std::vector<int>& want, std::vector<int>& st, acac_step_info* info) {
    if (h->mixed) nks<float>(h, want, st, info);
    else nks<double>(h, want, st, info);
}

// Energy and mass (Eqs. relations, freeenergy) of the members of mask `slot` (slot < 0:
// all) at X; bad[m] != 0 when some u + v or u - v of the member lies outside [0, 1].
void energy_members(acac_handle* h, int slot, const double* X, std::vector<double>& e, std::vector<double>& ms,
                    std::vector<int>& bad) {
    const Members mb = slot < 0 ? all_members(h) : on_mask(h, slot);
    CU(cudaMemsetAsync(h->flags, 0, sizeof(int) * h->B, h->stream));
    KLA(ACAC_K_ENERGY, 16.0 * h->N, 0.0, launch_energy(h->g, h->k, X, red_to(h, h->red), h->flags, h->stream, mb));
    fetch_flags(h);
    read_member_scalars(h, 0, 2);
    e.resize(h->B);
    ms.resize(h->B);
    bad.resize(h->B);
    for (int m = 0; m < h->B; ++m) {
        e[m] = h->host[2 * m];
        ms[m] = h->host[2 * m + 1];
        bad[m] = h->host_flags[m];
    }
}

// One accepted time step of every member (fields u, v: member m at m * N), with the
// adaptive step of Sec. 3.2: the predictor of Eq. sencondt from the last two states, and
// on divergence dt / sqrt(2) and eta doubled, retried until it converges or dt drops
// below dt_min.  The members retry independently (those done wait); info[m] per member.
// Returns the first failing status in member order.
int step_members(acac_handle* h, double* u, double* v, acac_step_info* info_out) {
    const int B = h->B;
    const size_t N = h->N;
    const long long n2 = 2 * (long long)N;
    std::vector<acac_step_info> info(B);
    memset(info.data(), 0, sizeof(acac_step_info) * B);
    const bool adaptive = h->p.dt_mode == ACAC_DT_ADAPTIVE;
    std::vector<double> dt(B, h->p.dt0);
    std::vector<int> prev(B);
    for (int m = 0; m < B; ++m) prev[m] = adaptive && h->have_prev[m];
    // U^n into X0 and, for the predictor, ||U^n - U^{n-1}||^2 in the same pass (members
    // without a previous state get a sum they do not read)
    KLA(ACAC_K_VECTOR, (any_of(prev) ? 48.0 : 32.0) * N, 0.0,
        launch_pack_state(u, v, h->X0, any_of(prev) ? h->Xprev : nullptr, (long long)N, red_to(h, h->red),
                          h->stream, all_members(h)));
    if (any_of(prev)) {
        read_member_scalars(h, 0, 1);
        for (int m = 0; m < B; ++m) {
            if (!prev[m]) continue;
            const double xd = sqrt(h->host[m]) / h->dt_prev[m];
            dt[m] = std::max(h->p.dt_min, h->p.dt_max / sqrt(1.0 + h->eta[m] * xd * xd));
        }
    }
    std::vector<int> pending(B, 1), stv(B, ACAC_OK), st;
    std::vector<double> e, ms;
    std::vector<int> bad;
    while (any_of(pending)) {
        for (int m = 0; m < B; ++m) {
            h->mk[m].dt = dt[m];
            h->mk[m].lam = 1.0;
        }
        write_members_any(h);
        nks_dispatch(h, pending, st, info.data());
        std::vector<int> ok(B, 0);
        for (int m = 0; m < B; ++m) {
            if (!pending[m]) continue;
            if (st[m] == ACAC_OK) {
                ok[m] = 1;
                pending[m] = 0;
            } else if (st[m] == ACAC_E_DIVERGED && adaptive) {
                info[m].divergences++;
                dt[m] = dt[m] / sqrt(2.0);
                h->eta[m] *= 2.0;
                if (dt[m] < h->p.dt_min) {
                    stv[m] = ACAC_E_DT_UNDERFLOW;
                    pending[m] = 0;
                }
            } else {
                if (st[m] == ACAC_E_DIVERGED) info[m].divergences++;
                stv[m] = st[m];
                pending[m] = 0;
            }
        }
        if (!any_of(ok)) continue;
        // accepted members: U^{n+1} out, U^n kept for the next predictor, energy and mass
        set_mask(h, MK_AUX, ok);
        const Members ma = on_mask(h, MK_AUX);
        // U^n becomes the predictor's previous state: when every member is accepted in this
        // round the buffers trade places (X0 is refilled by the next step), else a copy
        if (std::all_of(ok.begin(), ok.end(), [](int o) { return o != 0; })) std::swap(h->X0, h->Xprev);
        else KLA(ACAC_K_VECTOR, 32.0 * N, 0.0, launch_copy_members(h->X0, h->Xprev, n2, h->stream, ma));
        KLA(ACAC_K_VECTOR, 32.0 * N, 0.0, launch_pack_members(u, v, h->X, (long long)N, 0, h->stream, ma));
        energy_members(h, MK_AUX, h->X, e, ms, bad);
        for (int m = 0; m < B; ++m) {
            if (!ok[m]) continue;
            h->dt_prev[m] = dt[m];
            h->t[m] += dt[m];
            h->nstep[m]++;
            h->have_prev[m] = 1;
            info[m].energy = e[m];
            info[m].mass = ms[m];
            info[m].dt = dt[m];
            info[m].t = h->t[m];
        }
    }
    int first = ACAC_OK;
    for (int m = 0; m < B; ++m) {
        info[m].eta = h->eta[m];
        info[m].status = stv[m];
        if (first == ACAC_OK && stv[m] != ACAC_OK) first = stv[m];
    }
    if (info_out) memcpy(info_out, info.data(), sizeof(acac_step_info) * B);
    return first;
}

// ---------------------------------------------------------------- adjoint
// Reverse-mode derivative of the fixed-dt implicit step F(U^{n+1}, U^n; p) = 0:
//   J1^T mu = lambda^{n+1},  lambda^n = -J0^T mu,  dL/dp += -mu^T dF/dp,
// J1 = dF/dU^{n+1}, J0 = dF/dU^n at (U^{n+1}, U^n).  J1^T is formed by transposing the
// assembled stencil matrix, so GMRES uses the assembled product and the Schwarz/ILU(0)
// preconditioner factored from the subdomain blocks of J1^T.  FP64 handles only.

size_t stencil_values(const acac_handle* h) { return (size_t)(h->g.dim == 3 ? NSLOT3 : NSLOT) * 4 * h->N; }

void adjoint_buffers(acac_handle* h) {
    if (!h->adj) dmalloc(&h->adj, 8 * 2 * h->N * 4);
    if (!h->adjJ) dmalloc(&h->adjJ, stencil_values(h) * h->ksz);
}

// Linearisation at (X1, h->X0): pass A into G (flags: domain) and the cache of
// dF/dX1 (wrt_x0 = 0) or dF/dX0 (1), then the assembled matrix into h->adjJ and its
// transpose into h->J.
void assemble_transposed(acac_handle* h, const double* X1, double dt, int wrt_x0) {
    double* J = (double*)h->adjJ;
    KLA(ACAC_K_LINEARIZE, 56.0 * h->N + 56.0 * h->N, 0.0,
        launch_linearize<double>(h->g, h->k, X1, h->X0, h->G, cache_of<double>(h), h->stream, wrt_x0));
    // -dt puts -1/dt on the diagonal of dF/dX0
    set_dt0(h, wrt_x0 ? -dt : dt);
    KLA(ACAC_K_ASSEMBLE, 8.0 * 59.0 * h->N, 0.0,
        launch_assemble<double>(h->g, (const JacK<double>*)h->jk_dev, cache_of<double>(h), J, h->stream));
    set_dt0(h, dt);
    KLA(ACAC_K_VECTOR, 8.0 * 2.0 * stencil_values(h), 0.0, launch_transpose<double>(h->g, J, (double*)h->J, h->stream));
    h->jpacked = false;
}

// One adjoint step at (X1, X0) (device, 2N each).  lam_in = lambda^{n+1}; lam_out
// (may alias lam_in) receives lambda^n; grad[0..3] += -mu^T dF/d(alpha, beta, theta, gamma).
int adjoint_step(acac_handle* h, const double* X1, const double* X0, double dt, const double* lam_in,
                 double* lam_out, double* grad, double rtol, int* its) {
    const long long n2 = 2 * (long long)h->N;
    double* mu = h->adj;
    CU(cudaMemcpyAsync(h->X0, X0, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
    set_dt0(h, dt);
    eval_residual(h, -1, X1, false);
    if (h->fl[0] & 1) return ACAC_E_DOMAIN;
    // J1^T mu = lambda^{n+1}
    assemble_transposed(h, X1, dt, 0);
    int st = factor<double>(h, all_members(h));
    if (st != ACAC_OK) return st;
    CU(cudaMemcpyAsync(h->b, lam_in, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
    const acac_params saved = h->p;
    h->p.jac_mode = ACAC_JAC_ASSEMBLED;   // products with the transposed matrix in h->J
    h->p.graphs = 0;                      // the captured iterations use the forward product
    h->p.gmres_rtol = rtol;
    h->p.gmres_atol = 0.0;
    std::vector<int> gst, gits;
    std::vector<double> gres;
    try {
        gmres<double>(h, std::vector<int>(1, 1), mu, gst, gits, gres, nullptr);
    } catch (Err e) {
        h->p = saved;
        throw;
    }
    h->p = saved;
    st = gst[0];
    if (its) *its += gits[0];
    if (st != ACAC_OK) return st;
    // -mu^T dF/dp
    CU(cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream));
    KLA(ACAC_K_VECTOR, 8.0 * 7.0 * h->N, 0.0,
        launch_param_grad(h->g, h->k, X1, h->X0, h->G, mu, red_to(h, h->red), h->flags, h->stream));
    read_scalars(h, 4);
    for (int i = 0; i < 4; ++i) grad[i] += h->host[i];
    // lambda^n = -J0^T mu
    assemble_transposed(h, X1, dt, 1);
    KLA(ACAC_K_SPMV, 8.0 * h->N * 56, 104.0 * h->N, launch_spmv<double>(h->g, (const double*)h->J, mu, h->tmpd, h->stream));
    KL(ACAC_K_VECTOR, launch_to_krylov<double>(h->tmpd, -1.0, lam_out, n2, h->stream));
    return ACAC_OK;
}

// L(X) and dL/dX (into lam), dL/dp explicit part into grad[0..3].
int loss_and_grad(acac_handle* h, const double* X, const double* target, double wE, double wM, double* loss,
                  double* lam, double* grad) {
    CU(cudaMemsetAsync(h->flags, 0, sizeof(int), h->stream));
    KLA(ACAC_K_ENERGY, 8.0 * 6.0 * h->N, 0.0,
        launch_loss_grad(h->g, h->k, X, target, wE, wM, lam, red_to(h, h->red), h->flags, h->stream));
    CU(cudaMemcpyAsync(h->host_flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    read_scalars(h, 5);
    if (loss) *loss = h->host[0];
    for (int i = 0; i < 4; ++i) grad[i] = h->host[1 + i];
    return *h->host_flags ? ACAC_E_DOMAIN : ACAC_OK;
}

// ---------------------------------------------------------------- Schwarz tables
void partition_1d(int n, int P, std::vector<int>& s, std::vector<int>& e) {
    int base = n / P, rem = n % P, pos = 0;
    for (int k = 0; k < P; ++k) {
        int w = base + (k < rem ? 1 : 0);
        s.push_back(pos);
        e.push_back(pos + w);
        pos += w;
    }
}

int build_subdomains(acac_handle* h) {
    const acac_params& p = h->p;
    const int d = p.ras_overlap;
    const int dim = p.dim;
    std::vector<int> st[3], en[3];
    for (int a = 0; a < dim; ++a) partition_1d(p.n[a], p.ras_parts[a], st[a], en[a]);
    if (dim == 2) { st[2] = {0}; en[2] = {1}; }
    const int pz = dim == 3 ? p.ras_parts[2] : 1;
    h->subs.clear();
    h->lev.clear();
    h->cells3.clear();
    h->pos3.clear();
    long long coef = 0, vec = 0;
    int maxcnt = 1;
    size_t maxpad = 0;
    for (int kz = 0; kz < pz; ++kz) {
        for (int ky = 0; ky < p.ras_parts[1]; ++ky) {
            for (int kx = 0; kx < p.ras_parts[0]; ++kx) {
                const int kk[3] = {kx, ky, kz};
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    const int s0 = st[a][kk[a]], e0 = en[a][kk[a]];
                    if (a >= dim) { lo[a] = 0; hi[a] = 1; continue; }
                    if (p.bc == ACAC_BC_PERIODIC) {
                        lo[a] = s0 - d; hi[a] = e0 + d;
                        if (hi[a] - lo[a] > p.n[a] - 2) return ACAC_E_ARG;   // box would wrap onto itself
                    } else {
                        lo[a] = std::max(0, s0 - d); hi[a] = std::min(p.n[a], e0 + d);
                    }
                }
                SubInfo sd;
                memset(&sd, 0, sizeof(sd));
                sd.ox = lo[0]; sd.oy = lo[1]; sd.oz = lo[2];
                sd.W = hi[0] - lo[0]; sd.H = hi[1] - lo[1]; sd.D = hi[2] - lo[2];
                sd.own_x0 = st[0][kx] - lo[0]; sd.own_x1 = en[0][kx] - lo[0];
                sd.own_y0 = st[1][ky] - lo[1]; sd.own_y1 = en[1][ky] - lo[1];
                sd.own_z0 = st[2][kz] - lo[2]; sd.own_z1 = en[2][kz] - lo[2];
                // the stencil's offsets keep their natural order only in boxes of >= 4 cells
                if (sd.W < 4 || sd.H < 4 || (dim == 3 && sd.D < 4)) return ACAC_E_ARG;
                if (sd.W > 250 || sd.H > 250 || sd.D > 250) return ACAC_E_ARG;
                sd.nlev = (sd.W - 1) + 2 * (sd.H - 1) + (dim == 3 ? 3 * (sd.D - 1) : 0) + 1;
                sd.lev_base = (int)h->lev.size();
                sd.coef_base = coef;
                sd.vec_base = vec;
                sd.cell_base = (long long)h->cells3.size();
                int acc = 0;
                if (dim == 2) {
                    for (int l = 0; l < sd.nlev; ++l) {
                        h->lev.push_back(acc);
                        int cnt = 0;
                        for (int j = 0; j < sd.H; ++j) {
                            int i = l - 2 * j;
                            if (i >= 0 && i < sd.W) ++cnt;
                        }
                        maxcnt = std::max(maxcnt, cnt);
                        acc += cnt;
                    }
                } else {
                    // level-ordered cell list and the position of every cell in its level
                    const size_t ncell = (size_t)sd.W * sd.H * sd.D;
                    const size_t base = h->cells3.size();
                    h->cells3.resize(base + ncell);
                    h->pos3.resize(base + ncell);
                    for (int l = 0; l < sd.nlev; ++l) {
                        h->lev.push_back(acc);
                        int cnt = 0;
                        for (int k = 0; k < sd.D; ++k)
                            for (int j = 0; j < sd.H; ++j) {
                                const int i = l - 2 * j - 3 * k;
                                if (i < 0 || i >= sd.W) continue;
                                h->cells3[base + acc + cnt] = i | (j << 10) | (k << 20);
                                h->pos3[base + (size_t)(k * sd.H + j) * sd.W + i] = cnt;
                                ++cnt;
                            }
                        maxcnt = std::max(maxcnt, cnt);
                        acc += cnt;
                    }
                }
                h->lev.push_back(acc);
                coef += (long long)acc * (dim == 2 ? NCOEF : NCOEF3);
                const size_t pad = dim == 2 ? (size_t)ras_pitch(sd.W) * (sd.H + 4)
                                            : (size_t)ras3_pitch(sd.W, (int)h->ksz) * (sd.H + 4) * (sd.D + 4);
                vec += (long long)pad;
                maxpad = std::max(maxpad, pad);
                h->subs.push_back(sd);
            }
        }
    }
    h->coef_count = coef;
    if (dim == 3) {
        // records of every grid cell: box cells before the box + lo[level] + position in the
        // level's packed cell list (at most 8 boxes per cell)
        const size_t ncell = (size_t)p.n[0] * p.n[1] * p.n[2];
        h->rec_of.assign(8 * ncell, -1);
        for (const SubInfo& sd : h->subs) {
            const long long base = sd.coef_base / NCOEF3;
            const size_t nbc = (size_t)sd.W * sd.H * sd.D;
            for (size_t t = 0; t < nbc; ++t) {
                const int pk = h->cells3[sd.cell_base + t];
                const int i = pk & 1023, j = (pk >> 10) & 1023, k = pk >> 20;
                int gx = sd.ox + i, gy = sd.oy + j, gz = sd.oz + k;
                gx = gx < 0 ? gx + p.n[0] : (gx >= p.n[0] ? gx - p.n[0] : gx);
                gy = gy < 0 ? gy + p.n[1] : (gy >= p.n[1] ? gy - p.n[1] : gy);
                gz = gz < 0 ? gz + p.n[2] : (gz >= p.n[2] ? gz - p.n[2] : gz);
                const size_t gc = ((size_t)gz * p.n[1] + gy) * p.n[0] + gx;
                const long long rec = base + (long long)t;   // the cell list is in level order
                int q = 0;
                while (q < 8 && h->rec_of[8 * gc + q] >= 0) ++q;
                if (q == 8 || rec > INT32_MAX) return ACAC_E_ARG;
                h->rec_of[8 * gc + q] = (int)rec;
            }
        }
    }
    if (dim == 2) {
        // records of every grid cell: box cells before the box + lo[level] + position
        h->rec_of.assign((size_t)4 * p.n[0] * p.n[1], -1);
        h->own_of.assign((size_t)p.n[0] * p.n[1], 0);
        for (const SubInfo& sd : h->subs) {
            const long long base = sd.coef_base / NCOEF;
            for (int l = 0; l < sd.nlev; ++l) {
                const int t = l - sd.W + 2;
                const int jmin = t > 0 ? t / 2 : 0;
                for (int j = jmin; j < sd.H; ++j) {
                    const int i = l - 2 * j;
                    if (i < 0) break;
                    int gx = sd.ox + i, gy = sd.oy + j;
                    gx = gx < 0 ? gx + p.n[0] : (gx >= p.n[0] ? gx - p.n[0] : gx);
                    gy = gy < 0 ? gy + p.n[1] : (gy >= p.n[1] ? gy - p.n[1] : gy);
                    const size_t gc = (size_t)gy * p.n[0] + gx;
                    const long long rec = base + h->lev[sd.lev_base + l] + (j - jmin);
                    int q = 0;
                    while (q < 4 && h->rec_of[4 * gc + q] >= 0) ++q;
                    if (q == 4 || rec > INT32_MAX) return ACAC_E_ARG;   // at most 4 boxes per cell in 2D
                    h->rec_of[4 * gc + q] = (int)rec;
                    if (i >= sd.own_x0 && i < sd.own_x1 && j >= sd.own_y0 && j < sd.own_y1)
                        h->own_of[gc] = (unsigned char)q;
                }
            }
        }
    }
    int maxlev = 0;
    for (auto& sd : h->subs) maxlev = std::max(maxlev, sd.nlev);
    h->ras_maxlev = maxlev;
    h->ras_maxcnt = maxcnt;
    h->ras_maxpad = maxpad;
    h->nbox = (double)(coef / (dim == 2 ? NCOEF : NCOEF3));
    h->ras_threads = std::max(64, ((2 * maxcnt + 31) / 32) * 32);
    if (dim == 3) h->ras_threads = std::min(h->ras_threads, 512);
    if (h->ras_threads > 1024) h->ras_threads = 1024;
    h->ras_smem = maxpad * 2 * h->ksz;
    return ACAC_OK;
}

}  // namespace

acac::Geom acac::make_geom(const acac_params* p) {
    Geom g;
    memset(&g, 0, sizeof(g));
    g.nx = p->n[0]; g.ny = p->n[1]; g.bc = p->bc;
    g.dim = p->dim;
    g.nz = p->dim == 3 ? p->n[2] : 1;
    g.N = g.nx * g.ny * g.nz;
    g.hz = p->dim == 3 ? p->L[2] / p->n[2] : 1.0;
    g.ihz2 = p->dim == 3 ? 1.0 / (g.hz * g.hz) : 0.0;
    g.ihz2f = (float)g.ihz2;
    g.hx = p->L[0] / p->n[0]; g.hy = p->L[1] / p->n[1];
    g.ihx2 = 1.0 / (g.hx * g.hx); g.ihy2 = 1.0 / (g.hy * g.hy);
    g.ihx2f = (float)g.ihx2; g.ihy2f = (float)g.ihy2;
    g.hihx2 = 0.5 * g.ihx2; g.hihy2 = 0.5 * g.ihy2; g.hihz2 = 0.5 * g.ihz2;
    g.hihx2f = (float)g.hihx2; g.hihy2f = (float)g.hihy2; g.hihz2f = (float)g.hihz2;
    g.vol = g.hx * g.hy * (p->dim == 3 ? g.hz : 1.0);
    g.iso = g.ihx2 == g.ihy2 && (p->dim == 2 || g.ihz2 == g.ihx2);
    return g;
}

int acac::validate_params(const acac_params* p) {
    if (!p) return ACAC_E_ARG;
    if (p->dim != 2 && p->dim != 3) return ACAC_E_ARG;
    if (p->n[0] < 4 || p->n[1] < 4 || (p->dim == 3 && p->n[2] < 4)) return ACAC_E_ARG;
    if ((long long)p->n[0] * p->n[1] * (p->dim == 3 ? p->n[2] : 1) > (1LL << 30)) return ACAC_E_ARG;
    if (!(p->L[0] > 0 && p->L[1] > 0 && (p->dim == 2 || p->L[2] > 0))) return ACAC_E_ARG;
    if (p->dim == 3 && (p->ras_parts[2] < 1 || p->ras_parts[2] > p->n[2])) return ACAC_E_ARG;
    if (p->dim == 3 && p->bc == ACAC_BC_PERIODIC && p->ras_parts[2] < 2) return ACAC_E_ARG;
    if (p->bc != ACAC_BC_PERIODIC && p->bc != ACAC_BC_NEUMANN) return ACAC_E_ARG;
    if (!(p->alpha > 0 && p->beta > 0 && p->theta > 0 && p->gamma > 0 && p->rho > 0)) return ACAC_E_ARG;
    if (p->taylor_S < 1 || p->taylor_S > MAX_S) return ACAC_E_ARG;
    if (p->dt_mode != ACAC_DT_FIXED && p->dt_mode != ACAC_DT_ADAPTIVE) return ACAC_E_ARG;
    if (!(p->dt0 > 0)) return ACAC_E_ARG;
    if (p->dt_mode == ACAC_DT_ADAPTIVE && !(p->dt_min > 0 && p->dt_max >= p->dt_min && p->eta0 > 0))
        return ACAC_E_ARG;
    if (!(p->newton_rtol >= 0 && p->newton_atol >= 0) || p->newton_maxit < 1) return ACAC_E_ARG;
    if (!(p->gmres_rtol >= 0 && p->gmres_atol >= 0) || p->gmres_maxit < 1) return ACAC_E_ARG;
    if (p->gmres_restart < 1 || p->gmres_restart > MAX_RESTART) return ACAC_E_ARG;
    if (p->ras_parts[0] < 1 || p->ras_parts[1] < 1 || p->ras_parts[0] > p->n[0] || p->ras_parts[1] > p->n[1])
        return ACAC_E_ARG;
    if (p->bc == ACAC_BC_PERIODIC && (p->ras_parts[0] < 2 || p->ras_parts[1] < 2)) return ACAC_E_ARG;
    if (p->ras_overlap < 0) return ACAC_E_ARG;
    if (p->ras_type < 0 || p->ras_type > 2) return ACAC_E_ARG;
    if (p->precision != ACAC_FP64 && p->precision != ACAC_MIXED) return ACAC_E_ARG;
    if (p->jac_mode != ACAC_JAC_MATFREE && p->jac_mode != ACAC_JAC_ASSEMBLED) return ACAC_E_ARG;
    if (p->batch < 1 || p->batch > ACAC_MAX_BATCH) return ACAC_E_ARG;
    if (p->graphs != 0 && p->graphs != 1) return ACAC_E_ARG;
    if (p->ras_window < 0 || p->ras_window > 2) return ACAC_E_ARG;
    if (p->subdomain_solver < ACAC_SUB_ILU0 || p->subdomain_solver > ACAC_SUB_LU) return ACAC_E_ARG;
    if (p->subdomain_solver != ACAC_SUB_ILU0) {
        // the factorizations with fill hold a symbolic pattern per box shape on the host and a
        // column map per warp in shared memory: the largest box (ceil(n / P) + 2 delta cells
        // per axis, at most n) may hold 250 x 250 cells
        long long cells = 1;
        for (int a = 0; a < p->dim; ++a) {
            long long w = (p->n[a] + p->ras_parts[a] - 1) / p->ras_parts[a] + 2LL * p->ras_overlap;
            cells *= w < p->n[a] ? w : p->n[a];
        }
        if (cells > 250LL * 250) return ACAC_E_ARG;
    }
    return ACAC_OK;
}

namespace {

// Patterns, dependency levels and device tables of the subdomain solves with fill: one
// symbolic factorization per distinct box shape, values and pivot inverses per box.
void build_sparse(acac_handle* h) {
    const acac_params& p = h->p;
    const int fill = p.subdomain_solver == ACAC_SUB_LU ? -1 : p.subdomain_solver;
    std::vector<SparseBox> boxes;
    std::vector<long long> keys;
    long long blk = 0, cells = 0;
    for (const SubInfo& sd : h->subs) {
        const long long key = ((long long)sd.W << 40) | ((long long)sd.H << 20) | (long long)sd.D;
        int id = (int)(std::find(keys.begin(), keys.end(), key) - keys.begin());
        if (id == (int)keys.size()) {
            keys.push_back(key);
            h->sshape.push_back(build_sparse_shape(p.dim, sd.W, sd.H, sd.D, fill));
        }
        boxes.push_back(SparseBox{id, blk, cells});
        blk += h->sshape[id].ptr.back();
        cells += h->sshape[id].n;
    }
    h->sblocks = blk;
    h->scells = cells;
    // integer tables of all shapes in one device array
    std::vector<int> ints;
    struct Off8 { size_t o[8]; };
    std::vector<Off8> offs;
    int band = 0, width = 1, maxn = 0;
    for (const SparseShape& S : h->sshape) {
        Off8 o;
        const std::vector<int>* parts[8] = {&S.ptr, &S.col, &S.diag, &S.slot_pos, &S.flev_ptr, &S.flev_rows,
                                            &S.blev_ptr, &S.blev_rows};
        for (int q = 0; q < 8; ++q) {
            o.o[q] = ints.size();
            ints.insert(ints.end(), parts[q]->begin(), parts[q]->end());
            ints.resize((ints.size() + 3) & ~(size_t)3);
        }
        offs.push_back(o);
        band = std::max(band, S.band);
        maxn = std::max(maxn, S.n);
        for (size_t l = 0; l + 1 < S.flev_ptr.size(); ++l) width = std::max(width, S.flev_ptr[l + 1] - S.flev_ptr[l]);
        for (size_t l = 0; l + 1 < S.blev_ptr.size(); ++l) width = std::max(width, S.blev_ptr[l + 1] - S.blev_ptr[l]);
    }
    dmalloc(&h->sint_dev, ints.size() * sizeof(int));
    CU(cudaMemcpy(h->sint_dev, ints.data(), ints.size() * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<SparseShapeDev> sd(h->sshape.size());
    for (size_t t = 0; t < sd.size(); ++t) {
        const SparseShape& S = h->sshape[t];
        const int* b = h->sint_dev;
        sd[t] = SparseShapeDev{b + offs[t].o[0], b + offs[t].o[1], b + offs[t].o[2], b + offs[t].o[3],
                               b + offs[t].o[4], b + offs[t].o[5], b + offs[t].o[6], b + offs[t].o[7],
                               S.n, S.band, (int)S.flev_ptr.size() - 1, (int)S.blev_ptr.size() - 1, S.contig};
    }
    dmalloc(&h->sshape_dev, sd.size() * sizeof(SparseShapeDev));
    CU(cudaMemcpy(h->sshape_dev, sd.data(), sd.size() * sizeof(SparseShapeDev), cudaMemcpyHostToDevice));
    dmalloc(&h->sbox_dev, boxes.size() * sizeof(SparseBox));
    CU(cudaMemcpy(h->sbox_dev, boxes.data(), boxes.size() * sizeof(SparseBox), cudaMemcpyHostToDevice));
    auto r64 = [](long long e) { return (e + 63) / 64 * 64; };
    h->mb.cfs = r64(blk * 4);
    h->mb.rgs = r64(cells * 4);
    dmalloc(&h->sval, (size_t)h->mb.cfs * h->B * h->ksz);
    dmalloc(&h->sdinv, (size_t)h->mb.rgs * h->B * h->ksz);
    // apply: 8 warps, one per row of a dependency level (the whole block on a level of a
    // single row).  Factorization: 32 warps on the rows in natural order when positions
    // are arithmetic, else 16 (fewer if their maps do not fit shared memory)
    h->s_threads = 256;
    (void)width;
    bool contig = true;
    for (const SparseShape& S : h->sshape) contig = contig && S.contig;
    h->s_use_map = contig ? 0 : 1;
    const size_t words = (size_t)((maxn + 31) / 32 + 3) / 4 * 4;
    int fw = contig ? 32 : 16;
    while (fw > 1 && (words + (contig ? 0 : (size_t)fw * (2 * band + 1))) * sizeof(int) > 200 * 1024) fw /= 2;
    h->s_fthreads = 32 * fw;
    h->s_fsmem = (words + (contig ? 0 : (size_t)fw * (2 * band + 1))) * sizeof(int);
    const size_t vec = (size_t)maxn * 2 * h->ksz;
    if (vec <= 96 * 1024) {
        h->s_asmem = vec;
    } else {
        h->s_asmem = 0;
        h->mb.ss = r64(cells * 2);
        dmalloc(&h->sy, (size_t)h->mb.ss * h->B * h->ksz);
    }
    if (p.ras_type != ACAC_RAS_LEFT) {
        // the box cells of every grid cell (natural order within each box), for the additive
        // extensions' fixed-order sums
        const int rpc = p.dim == 3 ? 8 : 4;
        const size_t ncell = h->N;
        std::vector<int> map(rpc * ncell, -1);
        for (size_t bi = 0; bi < h->subs.size(); ++bi) {
            const SubInfo& sd = h->subs[bi];
            const long long base = boxes[bi].cell_base;
            const int D = p.dim == 3 ? sd.D : 1;
            for (int k = 0; k < D; ++k)
                for (int j = 0; j < sd.H; ++j)
                    for (int i = 0; i < sd.W; ++i) {
                        auto wrap = [&](int x, int n) {
                            return p.bc == ACAC_BC_PERIODIC ? (x < 0 ? x + n : (x >= n ? x - n : x))
                                                            : (x < 0 ? 0 : (x >= n ? n - 1 : x));
                        };
                        const int gx = wrap(sd.ox + i, p.n[0]), gy = wrap(sd.oy + j, p.n[1]);
                        const int gz = p.dim == 3 ? wrap(sd.oz + k, p.n[2]) : 0;
                        const size_t gc = ((size_t)gz * p.n[1] + gy) * p.n[0] + gx;
                        const long long rec = base + ((long long)k * sd.H + j) * sd.W + i;
                        int q = 0;
                        while (q < rpc && map[rpc * gc + q] >= 0) ++q;
                        if (q == rpc || rec > INT32_MAX) throw Err{ACAC_E_ARG};
                        map[rpc * gc + q] = (int)rec;
                    }
        }
        dmalloc(&h->srec_of_dev, map.size() * sizeof(int));
        CU(cudaMemcpy(h->srec_of_dev, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    for (SparseShape& S : h->sshape) {   // the device holds what the kernels need
        S.col.clear(); S.col.shrink_to_fit();
        S.slot_pos.clear(); S.slot_pos.shrink_to_fit();
    }
}

void free_all(acac_handle* h) {
    void* bufs[] = {h->X, h->X0, h->Xprev, h->Xt, h->F, h->S, h->G, h->b, h->r, h->tmpd, h->stage, h->lap0,
                    h->mk_dev, h->masks, h->ghead_dev, h->gwork_dev, h->kcnt_dev, h->V, h->Zb, h->w,
                    h->kt, h->jtmp, h->cache, h->J, h->coef, h->gscratch, h->partial, h->red, h->flags,
                    h->counter, h->subs_dev, h->lev_dev, h->cells3_dev, h->pos3_dev, h->rec_of_dev, h->own_of_dev,
                    h->rg, h->Jp,
                    h->sshape_dev, h->sbox_dev, h->sint_dev, h->sval, h->sdinv, h->sy, h->srec_of_dev, h->zb};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (h->host) cudaFreeHost(h->host);
    if (h->host_flags) cudaFreeHost(h->host_flags);
    if (h->jk_dev) cudaFree(h->jk_dev);
    if (h->adj) cudaFree(h->adj);
    if (h->adjJ) cudaFree(h->adjJ);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->stream) cudaStreamDestroy(h->stream);
}

}  // namespace


// ====================================================================== C ABI
extern "C" {

void acac_default_params(acac_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->dim = 2;
    p->n[0] = 64; p->n[1] = 64; p->n[2] = 1;
    p->L[0] = 1.0; p->L[1] = 1.0; p->L[2] = 1.0;
    p->bc = ACAC_BC_PERIODIC;
    p->alpha = 3.0; p->beta = 1.0; p->theta = 0.3; p->gamma = 1e-3; p->rho = 1.0;
    p->taylor_S = 10;
    p->dt_mode = ACAC_DT_FIXED;
    p->dt0 = 1e-3; p->dt_min = 1e-5; p->dt_max = 1e-1; p->eta0 = 1e4;
    p->newton_rtol = 1e-8; p->newton_atol = 1e-13; p->newton_maxit = 20;
    p->gmres_rtol = 1e-6; p->gmres_atol = 1e-14; p->gmres_restart = 30; p->gmres_maxit = 500;
    p->ras_parts[0] = 4; p->ras_parts[1] = 4; p->ras_parts[2] = 1;
    p->ras_overlap = 1;
    p->ras_type = ACAC_RAS_LEFT;
    p->ilu_reuse = 1;
    p->precision = ACAC_FP64;
    p->jac_mode = ACAC_JAC_MATFREE;
    p->batch = 1;
    p->cgs_refine = 1;
    p->graphs = 1;
}

const char* acac_status_string(int s) {
    switch (s) {
        case ACAC_OK: return "ok";
        case ACAC_E_ARG: return "invalid argument";
        case ACAC_E_CUDA: return "CUDA error";
        case ACAC_E_DOMAIN: return "state outside the admissible set";
        case ACAC_E_DIVERGED: return "Newton-Krylov-Schwarz solve diverged";
        case ACAC_E_DT_UNDERFLOW: return "time step fell below dt_min";
        case ACAC_E_TIMEOUT: return "device wait timed out";
        case ACAC_E_NOMEM: return "out of memory";
        default: return "unknown status";
    }
}

int acac_create(const acac_params* p, void* cuda_stream, acac_handle** out) {
    if (!out) return ACAC_E_ARG;
    *out = nullptr;
    int st = validate_params(p);
    if (st != ACAC_OK) return st;
    acac_handle* h = new (std::nothrow) acac_handle();
    if (!h) return ACAC_E_NOMEM;
    h->p = *p;
    h->user_stream = (cudaStream_t)cuda_stream;
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return ACAC_E_CUDA;
    }
    h->mixed = p->precision == ACAC_MIXED;
    h->ksz = h->mixed ? sizeof(float) : sizeof(double);
    h->N = (size_t)p->n[0] * p->n[1] * (p->dim == 3 ? p->n[2] : 1);
    h->g = make_geom(p);
    h->k = Coef{p->alpha, p->beta, p->theta, p->gamma, p->rho, p->taylor_S};
    const int B = h->B = p->batch;
    h->mk.assign(B, MemberK{p->alpha, p->beta, p->theta, p->gamma, p->rho, p->dt0, 1.0, 0.0});
    h->t.assign(B, 0.0);
    h->dt_prev.assign(B, 0.0);
    h->eta.assign(B, p->eta0);
    h->nstep.assign(B, 0);
    h->have_prev.assign(B, 0);
    h->fn.assign(B, 0.0);
    h->fl.assign(B, 0);
    for (auto& v : h->mask_host) v.assign(B, -1);   // nothing written yet
    st = build_subdomains(h);
    if (st != ACAC_OK) {
        cudaStreamDestroy(h->stream);
        delete h;
        return st;
    }
    try {
        const size_t N = h->N, n2 = 2 * N, ks = h->ksz, Bz = (size_t)B;
        // per-member strides, 64 elements aligned (256 bytes for doubles): every member's
        // buffers start where the single-problem kernels expect their alignment
        auto r64 = [](long long e) { return (e + 63) / 64 * 64; };
        Members& mb = h->mb;
        mb.count = B;
        mb.vs = r64((long long)n2);
        mb.gs = r64(3LL * (long long)N);
        mb.cs = r64(7LL * (long long)N);
        mb.js = r64((long long)(p->dim == 3 ? NSLOT3 : NSLOT) * 4 * (long long)N);
        mb.jps = r64(p->dim == 3 ? (h->coef_count / NCOEF3) * 4 * NSLOT3 : (h->coef_count / NCOEF) * 4 * NSLOT);
        mb.cfs = r64(h->coef_count);
        mb.rs = RS;
        mb.ps = (long long)(MAX_RESTART + 3) * red_grid((long long)n2);
        const size_t vz = (size_t)mb.vs * Bz;
        dmalloc(&h->X, vz * 8); dmalloc(&h->X0, vz * 8); dmalloc(&h->Xprev, vz * 8);
        dmalloc(&h->Xt, vz * 8); dmalloc(&h->F, vz * 8); dmalloc(&h->S, vz * 8);
        dmalloc(&h->G, (size_t)mb.gs * Bz * 8); dmalloc(&h->b, vz * 8); dmalloc(&h->r, vz * 8);
        dmalloc(&h->tmpd, vz * 8);
        dmalloc(&h->stage, n2 * Bz * 8);
        dmalloc(&h->lap0, vz * 8);
        dmalloc(&h->mk_dev, sizeof(MemberK) * Bz);
        dmalloc(&h->masks, sizeof(int) * MK_COUNT * Bz);
        dmalloc(&h->ghead_dev, sizeof(GmresHead) * Bz);
        dmalloc(&h->gwork_dev, sizeof(GmresWork) * Bz);
        dmalloc(&h->kcnt_dev, sizeof(int) * Bz);
        h->ldV = vz;
        dmalloc(&h->V, (size_t)(p->gmres_restart + 1) * h->ldV * ks);
        dmalloc(&h->Zb, (size_t)p->gmres_restart * h->ldV * ks);
        dmalloc(&h->w, vz * ks); dmalloc(&h->kt, vz * ks);
        dmalloc(&h->jtmp, (size_t)mb.gs * Bz * ks);
        dmalloc(&h->cache, (size_t)mb.cs * Bz * ks);
        dmalloc(&h->J, (size_t)mb.js * Bz * ks);
        dmalloc(&h->coef, (size_t)(p->subdomain_solver == ACAC_SUB_ILU0 ? mb.cfs * Bz : 1) * ks);
        int dev = 0;
        CU(cudaGetDevice(&dev));
        int optin = 0;
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (p->dim == 3) {
            // 3D apply: mbarriers | level table | record stages (TMA ring) | padded box vector
            // (shared memory when it fits, else global)
            auto r128 = [](size_t b) { return (b + 127) / 128 * 128; };
            RasLaunch& L = h->ras_launch;
            L.window = 0;
            L.stage_off = (int)(16 * RAS_MAXBUF + r128((size_t)(h->ras_maxlev + 1) * 4));
            L.stage_elems = (CREC3 * h->ras_maxcnt + 31) / 32 * 32;
            L.threads = 32 * ((2 * h->ras_maxcnt + 31) / 32) + 32;
            const size_t vec_bytes = r128(h->ras_maxpad * 2 * ks);
            const size_t stage_bytes = (size_t)L.stage_elems * ks;
            const size_t cap = (size_t)optin - 2048, half = 113 * 1024;
            // at least 4 stages in flight (fewer leave each level waiting on its copy): the
            // vector in shared memory at two CTAs per SM, else at one CTA per SM, else in
            // global scratch at two CTAs per SM
            bool vec_in_smem = true;
            if (L.stage_off + vec_bytes + 4 * stage_bytes <= half) {
                L.nbuf = (int)std::min<size_t>(RAS_MAXBUF, (half - L.stage_off - vec_bytes) / stage_bytes);
            } else if (L.stage_off + vec_bytes + 4 * stage_bytes <= cap) {
                L.nbuf = (int)std::min<size_t>(RAS_MAXBUF, (cap - L.stage_off - vec_bytes) / stage_bytes);
            } else {
                vec_in_smem = false;
                L.nbuf = (int)std::max<size_t>(2, std::min<size_t>(RAS_MAXBUF, (half - L.stage_off) / stage_bytes));
            }
            L.vec_off = (int)(L.stage_off + (size_t)L.nbuf * L.stage_elems * ks);
            L.smem_bytes = L.vec_off + (vec_in_smem ? vec_bytes : 0);
            if (!vec_in_smem) {
                size_t tot = 0;
                for (auto& sd : h->subs) tot += (size_t)ras3_pitch(sd.W, (int)ks) * (sd.H + 4) * (sd.D + 4);
                mb.ss = r64((long long)tot * 2);
                dmalloc(&h->gscratch, (size_t)mb.ss * Bz * ks);
            }
        } else {
        // shared-memory plan of the Schwarz apply: mbarriers | level table | coefficient
        // stages | box vector.  Prefer a plan with two CTAs per SM.
            auto r128 = [](size_t b) { return (b + 127) / 128 * 128; };
            RasLaunch& L = h->ras_launch;
            L.stage_vec = 0;
            L.stage_off = (int)(16 * RAS_MAXBUF + r128((size_t)(h->ras_maxlev + 1) * 4));
            L.stage_elems = (CREC * h->ras_maxcnt + 31) / 32 * 32;
            L.threads = 32 * ((2 * h->ras_maxcnt + 31) / 32) + 32;
            const size_t vec_bytes = r128(h->ras_maxpad * 2 * ks);
            const size_t stage_bytes = (size_t)L.stage_elems * ks;
            const size_t cap = (size_t)optin - 2048;
            // The sweeps stream every level's coefficients once: keep as many stages in
            // flight per SM as shared memory allows (TMA latency is several us).  With
            // the box vector in shared memory, take two CTAs per SM when at least 3 stages
            // fit per CTA, else one CTA per SM with up to RAS_MAXBUF stages.
            bool vec_in_smem = false;
            const size_t half = 113 * 1024;
            const bool full_fits2 = L.stage_off + vec_bytes + 3 * stage_bytes <= half;
            // windowed apply (the last 5 levels in shared memory, the forward result in
            // global scratch) when the box vector does not fit two CTAs per SM, or on request
            L.window = p->ras_window == 1 || (p->ras_window == 0 && !full_fits2);
            int maxh = 0;
            for (auto& sd : h->subs) maxh = std::max(maxh, sd.H);
            L.win_cells = maxh + 4;   // rows per window slot
            if (L.window) {
                // a windowed stage also carries the level's right-hand side (2 values per cell,
                // copied in 16-byte chunks from a possibly unaligned start)
                L.stage_vec = L.stage_elems;
                L.stage_elems += (2 * h->ras_maxcnt + 8 + 31) / 32 * 32;
                // float: the right-hand side gathered per box cell (in record order), read by the
                // stages; 16 spare values for the chunked copies' overreach
                mb.rgs = r64((h->coef_count / NCOEF) * 2 + 16);
                if (ks == 4) dmalloc(&h->rg, (size_t)mb.rgs * Bz * ks);
                const size_t stage_bytes = (size_t)L.stage_elems * ks;
                // aim at three CTAs per SM with at least 4 stages each
                const size_t win_bytes = r128((size_t)5 * L.win_cells * 2 * ks);
                const size_t third = 74 * 1024;
                const size_t room = third > L.stage_off + win_bytes ? third - L.stage_off - win_bytes : 0;
                L.nbuf = (int)std::max<size_t>(4, std::min<size_t>(RAS_MAXBUF, room / stage_bytes));
                L.vec_off = (int)(L.stage_off + (size_t)L.nbuf * L.stage_elems * ks);
                L.smem_bytes = L.vec_off + win_bytes;
                size_t tot = 0;
                for (auto& sd : h->subs) tot += (size_t)ras_pitch(sd.W) * (sd.H + 4);
                mb.ss = r64((long long)tot * 2);
                dmalloc(&h->gscratch, (size_t)mb.ss * Bz * ks);
            } else if (L.stage_off + vec_bytes + 3 * stage_bytes <= half) {
                L.nbuf = (int)std::min<size_t>(RAS_MAXBUF, (half - L.stage_off - vec_bytes) / stage_bytes);
                vec_in_smem = true;
            } else if (L.stage_off + vec_bytes + 4 * stage_bytes <= cap) {
                L.nbuf = (int)std::min<size_t>(RAS_MAXBUF, (cap - L.stage_off - vec_bytes) / stage_bytes);
                vec_in_smem = true;
            } else {
                L.nbuf = (int)std::min<size_t>(RAS_MAXBUF, (cap - L.stage_off) / stage_bytes);
            }
            if (!L.window) {
                L.vec_off = (int)(L.stage_off + (size_t)L.nbuf * L.stage_elems * ks);
                L.smem_bytes = L.vec_off + (vec_in_smem ? vec_bytes : 0);
                if (!vec_in_smem) {
                    size_t tot = 0;
                    for (auto& sd : h->subs) tot += (size_t)ras_pitch(sd.W) * (sd.H + 4);
                    mb.ss = r64((long long)tot * 2);
                dmalloc(&h->gscratch, (size_t)mb.ss * Bz * ks);
                }
            }
        }
        dmalloc(&h->partial, (size_t)mb.ps * Bz * 8);
        dmalloc(&h->red, (size_t)RS * Bz * 8);
        dmalloc(&h->flags, sizeof(int) * 2 * Bz);
        CU(cudaMemset(h->flags, 0, sizeof(int) * 2 * Bz));
        dmalloc(&h->counter, sizeof(unsigned) * Bz);
        CU(cudaMemset(h->counter, 0, sizeof(unsigned) * Bz));
        dmalloc(&h->jk_dev, sizeof(JacK<double>) * Bz);
        mb.k = h->mk_dev;
        CU(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
        CU(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
        CU(cudaMallocHost((void**)&h->host, (size_t)RS * Bz * 8));
        CU(cudaMallocHost((void**)&h->host_flags, sizeof(int) * 3 * Bz));
        dmalloc(&h->subs_dev, h->subs.size() * sizeof(SubInfo));
        dmalloc(&h->lev_dev, h->lev.size() * sizeof(int));
        dmalloc(&h->cells3_dev, std::max<size_t>(1, h->cells3.size()) * sizeof(int));
        dmalloc(&h->pos3_dev, std::max<size_t>(1, h->pos3.size()) * sizeof(int));
        if (!h->cells3.empty()) {
            CU(cudaMemcpy(h->cells3_dev, h->cells3.data(), h->cells3.size() * sizeof(int), cudaMemcpyHostToDevice));
            CU(cudaMemcpy(h->pos3_dev, h->pos3.data(), h->pos3.size() * sizeof(int), cudaMemcpyHostToDevice));
        }
        CU(cudaMemcpy(h->subs_dev, h->subs.data(), h->subs.size() * sizeof(SubInfo), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(h->lev_dev, h->lev.data(), h->lev.size() * sizeof(int), cudaMemcpyHostToDevice));
        dmalloc(&h->rec_of_dev, h->rec_of.size() * sizeof(int));
        CU(cudaMemcpy(h->rec_of_dev, h->rec_of.data(), h->rec_of.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (!h->own_of.empty()) {
            dmalloc(&h->own_of_dev, h->own_of.size());
            CU(cudaMemcpy(h->own_of_dev, h->own_of.data(), h->own_of.size(), cudaMemcpyHostToDevice));
            h->own_of.clear();
            h->own_of.shrink_to_fit();
        }
        dmalloc(&h->Jp, (size_t)mb.jps * Bz * h->ksz);
        h->rec_of.clear();
        h->rec_of.shrink_to_fit();
        if (p->subdomain_solver != ACAC_SUB_ILU0) build_sparse(h);
        if (p->ras_type != ACAC_RAS_LEFT) {
            // additive extensions: every box cell's two values, summed per grid cell afterwards
            const long long bcells = p->subdomain_solver != ACAC_SUB_ILU0 ? h->scells
                                   : h->coef_count / (p->dim == 3 ? NCOEF3 : NCOEF);
            mb.zs = r64(2 * bcells);
            dmalloc(&h->zb, (size_t)mb.zs * Bz * ks);
        }
        CU(set_taylor_constants(p->taylor_S));
        std::vector<int> ones(B, 1);
        set_mask(h, MK_NEWTON, ones);
        write_members_any(h);
        CU(cudaStreamSynchronize(h->stream));
    } catch (Err e) {
        free_all(h);
        delete h;
        return e.code;
    }
    *out = h;
    return ACAC_OK;
}

void acac_destroy(acac_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto& p : h->pending) {
        if (p.owned_by_graph) continue;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
    free_graphs(h);
    free_all(h);
    delete h;
}

int acac_log(const double* x, double* y, long long n, void* cuda_stream) {
    if (!x || !y || n < 0) return ACAC_E_ARG;
    if (launch_table_log(x, y, n, (cudaStream_t)cuda_stream) != cudaSuccess) return ACAC_E_CUDA;
    return ACAC_OK;
}

int acac_profile(acac_handle* h, int enable) { return acac_profile_mask(h, enable ? 0xffffffffu : 0u); }

int acac_profile_mask(acac_handle* h, unsigned mask) {
    if (!h) return ACAC_E_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return ACAC_E_CUDA;
    try {
        prof_collect(h);
    } catch (Err e) {
        return e.code;
    }
    h->prof_on = mask != 0;
    h->prof_mask = mask;
    for (int i = 0; i < ACAC_NKERNEL; ++i) {
        h->launches[i] = 0;
        h->kernel_ms[i] = 0.0;
        h->kernel_bytes[i] = 0.0;
        h->kernel_flops[i] = 0.0;
    }
    return ACAC_OK;
}

int acac_kernel_stats(acac_handle* h, int kernel, long long* launches, double* total_ms, double* bytes,
                      double* flops) {
    if (!h || kernel < 0 || kernel >= ACAC_NKERNEL) return ACAC_E_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return ACAC_E_CUDA;
    try {
        prof_collect(h);
    } catch (Err e) {
        return e.code;
    }
    if (launches) *launches = h->launches[kernel];
    if (total_ms) *total_ms = h->kernel_ms[kernel];
    if (bytes) *bytes = h->kernel_bytes[kernel];
    if (flops) *flops = h->kernel_flops[kernel];
    return ACAC_OK;
}

int acac_set_coeffs(acac_handle* h, int member, double alpha, double beta, double theta, double gamma,
                    double rho) {
    if (!h) return ACAC_E_ARG;
    if (!(alpha > 0 && beta > 0 && theta > 0 && gamma > 0 && rho > 0)) return ACAC_E_ARG;
    if (member < 0 || member >= h->B) return ACAC_E_ARG;
    MemberK& q = h->mk[member];
    q.alpha = alpha; q.beta = beta; q.theta = theta; q.gamma = gamma; q.rho = rho;
    if (member == 0) {
        h->p.alpha = alpha; h->p.beta = beta; h->p.theta = theta; h->p.gamma = gamma; h->p.rho = rho;
        h->k = Coef{alpha, beta, theta, gamma, rho, h->p.taylor_S};
    }
    // on the device with the next step (write_members); single-problem calls write them
    // with their dt
    return ACAC_OK;
}

const char* acac_kernel_name(int kernel) {
    static const char* names[ACAC_NKERNEL] = {
        "residual_g", "residual_f", "linearize", "assemble", "spmv", "jvp_g", "jvp_f",
        "ras_factor", "ras_apply", "gs_dot", "gs_update", "repack", "vector", "energy"};
    return (kernel >= 0 && kernel < ACAC_NKERNEL) ? names[kernel] : "unknown";
}

int acac_residual(acac_handle* h, const double* X1, const double* X0, double dt, double* F, double* fnorm) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !X1 || !X0 || !F || !(dt > 0)) return ACAC_E_ARG;
    Join join(h);
    try {
        const size_t n2 = 2 * h->N;
        CU(cudaMemcpyAsync(h->X0, X0, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
        set_dt0(h, dt);
        eval_residual(h, -1, X1, false);
        CU(cudaMemcpyAsync(F, h->F, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        if (fnorm) *fnorm = h->fn[0];
        return (h->fl[0] & 1) ? ACAC_E_DOMAIN : ACAC_OK;
    } catch (Err e) {
        return e.code;
    }
}

// Linearise at X1 (pass A of the residual fills G, then the cache).
static int linearize_at(acac_handle* h, const double* X1, const double* X0, double dt) {
    const size_t n2 = 2 * h->N;
    CU(cudaMemcpyAsync(h->X0, X0, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
    set_dt0(h, dt);
    eval_residual(h, -1, X1, false);
    if (h->fl[0] & 1) return ACAC_E_DOMAIN;
    if (h->mixed)
        KL(ACAC_K_LINEARIZE, launch_linearize<float>(h->g, h->k, X1, h->X0, h->G, cache_of<float>(h), h->stream));
    else
        KL(ACAC_K_LINEARIZE, launch_linearize<double>(h->g, h->k, X1, h->X0, h->G, cache_of<double>(h), h->stream));
    return ACAC_OK;
}

int acac_jacobian(acac_handle* h, const double* X1, const double* X0, double dt, void* J) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !X1 || !X0 || !J || !(dt > 0)) return ACAC_E_ARG;
    Join join(h);
    try {
        int st = linearize_at(h, X1, X0, dt);
        if (st != ACAC_OK) return st;
        if (h->mixed)
            KL(ACAC_K_ASSEMBLE, launch_assemble<float>(h->g, (const JacK<float>*)h->jk_dev, cache_of<float>(h),
                                                       (float*)J, h->stream));
        else
            KL(ACAC_K_ASSEMBLE, launch_assemble<double>(h->g, (const JacK<double>*)h->jk_dev, cache_of<double>(h),
                                                        (double*)J, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        return ACAC_OK;
    } catch (Err e) {
        return e.code;
    }
}

int acac_spmv(acac_handle* h, const void* J, const void* w, void* y) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !J || !w || !y) return ACAC_E_ARG;
    Join join(h);
    try {
        if (h->mixed)
            KL(ACAC_K_SPMV, launch_spmv<float>(h->g, (const float*)J, (const float*)w, (float*)y, h->stream));
        else
            KL(ACAC_K_SPMV, launch_spmv<double>(h->g, (const double*)J, (const double*)w, (double*)y, h->stream));
        return ACAC_OK;
    } catch (Err e) {
        return e.code;
    }
}

int acac_jvp(acac_handle* h, const double* X1, const double* X0, double dt, const void* w, void* y) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !X1 || !X0 || !w || !y || !(dt > 0)) return ACAC_E_ARG;
    Join join(h);
    try {
        int st = linearize_at(h, X1, X0, dt);
        if (st != ACAC_OK) return st;
        if (h->mixed) jvp_action<float>(h, all_members(h), (const float*)w, (float*)y);
        else jvp_action<double>(h, all_members(h), (const double*)w, (double*)y);
        return ACAC_OK;
    } catch (Err e) {
        return e.code;
    }
}

int acac_ras_factor(acac_handle* h, const void* J) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !J) return ACAC_E_ARG;
    Join join(h);
    try {
        const size_t bytes = (size_t)(h->g.dim == 3 ? NSLOT3 : NSLOT) * 4 * h->N * h->ksz;
        if (J != h->J) CU(cudaMemcpyAsync(h->J, J, bytes, cudaMemcpyDeviceToDevice, h->stream));
        h->jpacked = false;
        return h->mixed ? factor<float>(h, all_members(h)) : factor<double>(h, all_members(h));
    } catch (Err e) {
        return e.code;
    }
}

int acac_ras_apply(acac_handle* h, const void* r, void* z) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !r || !z) return ACAC_E_ARG;
    Join join(h);
    try {
        if (h->mixed) precond<float>(h, all_members(h), (const float*)r, (float*)z);
        else precond<double>(h, all_members(h), (const double*)r, (double*)z);
        return ACAC_OK;
    } catch (Err e) {
        return e.code;
    }
}

int acac_gmres(acac_handle* h, const double* X1, const double* X0, double dt, const double* b, double* x,
               int* its, double* resid) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !X1 || !X0 || !b || !x || !(dt > 0)) return ACAC_E_ARG;
    Join join(h);
    try {
        int st = linearize_at(h, X1, X0, dt);
        if (st != ACAC_OK) return st;
        CU(cudaMemcpyAsync(h->b, b, 2 * h->N * 8, cudaMemcpyDeviceToDevice, h->stream));
        h->jpacked = false;
        const std::vector<int> one(1, 1);
        std::vector<int> gst(1, ACAC_OK), gits(1, 0);
        std::vector<double> gres(1, 0.0);
        if (h->mixed) {
            KL(ACAC_K_ASSEMBLE, launch_assemble<float>(h->g, (const JacK<float>*)h->jk_dev, cache_of<float>(h),
                                                       (float*)h->J, h->stream));
            st = factor<float>(h, all_members(h));
            if (st == ACAC_OK) gmres<float>(h, one, x, gst, gits, gres, nullptr);
        } else {
            KL(ACAC_K_ASSEMBLE, launch_assemble<double>(h->g, (const JacK<double>*)h->jk_dev, cache_of<double>(h),
                                                        (double*)h->J, h->stream));
            st = factor<double>(h, all_members(h));
            if (st == ACAC_OK) gmres<double>(h, one, x, gst, gits, gres, nullptr);
        }
        if (st == ACAC_OK) st = gst[0];
        if (its) *its = gits[0];
        if (resid) *resid = gres[0];
        return st;
    } catch (Err e) {
        return e.code;
    }
}

int acac_nks_solve(acac_handle* h, const double* U0, double dt, double* U1, acac_step_info* info) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !U0 || !U1 || !(dt > 0)) return ACAC_E_ARG;
    Join join(h);
    acac_step_info local;
    memset(&local, 0, sizeof(local));
    int st;
    try {
        CU(cudaMemcpyAsync(h->X0, U0, 2 * h->N * 8, cudaMemcpyDeviceToDevice, h->stream));
        set_dt0(h, dt);
        std::vector<int> sv;
        nks_dispatch(h, std::vector<int>(1, 1), sv, &local);
        st = sv[0];
        if (st == ACAC_OK) CU(cudaMemcpyAsync(U1, h->X, 2 * h->N * 8, cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaStreamSynchronize(h->stream));
    } catch (Err e) {
        st = e.code;
    }
    local.status = st;
    local.dt = dt;
    if (info) *info = local;
    return st;
}

int acac_jacobian_x0(acac_handle* h, const double* X1, const double* X0, double dt, void* J) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !X1 || !X0 || !J || !(dt > 0)) return ACAC_E_ARG;
    Join join(h);
    try {
        int st = linearize_at(h, X1, X0, dt);
        if (st != ACAC_OK) return st;
        if (h->mixed) {
            KL(ACAC_K_LINEARIZE, launch_linearize<float>(h->g, h->k, X1, h->X0, h->G, cache_of<float>(h), h->stream, 1));
            set_dt0(h, -dt);
            KL(ACAC_K_ASSEMBLE, launch_assemble<float>(h->g, (const JacK<float>*)h->jk_dev, cache_of<float>(h),
                                                       (float*)J, h->stream));
        } else {
            KL(ACAC_K_LINEARIZE, launch_linearize<double>(h->g, h->k, X1, h->X0, h->G, cache_of<double>(h), h->stream, 1));
            set_dt0(h, -dt);
            KL(ACAC_K_ASSEMBLE, launch_assemble<double>(h->g, (const JacK<double>*)h->jk_dev, cache_of<double>(h),
                                                        (double*)J, h->stream));
        }
        CU(cudaStreamSynchronize(h->stream));
        return ACAC_OK;
    } catch (Err e) {
        return e.code;
    }
}

int acac_spmv_t(acac_handle* h, const void* J, const void* w, void* y) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !J || !w || !y) return ACAC_E_ARG;
    Join join(h);
    try {
        adjoint_buffers(h);
        if (h->mixed) {
            KL(ACAC_K_VECTOR, launch_transpose<float>(h->g, (const float*)J, (float*)h->adjJ, h->stream));
            KL(ACAC_K_SPMV, launch_spmv<float>(h->g, (const float*)h->adjJ, (const float*)w, (float*)y, h->stream));
        } else {
            KL(ACAC_K_VECTOR, launch_transpose<double>(h->g, (const double*)J, (double*)h->adjJ, h->stream));
            KL(ACAC_K_SPMV, launch_spmv<double>(h->g, (const double*)h->adjJ, (const double*)w, (double*)y, h->stream));
        }
        return ACAC_OK;
    } catch (Err e) {
        return e.code;
    }
}

int acac_loss(acac_handle* h, const double* X, const double* target, double w_energy, double w_misfit,
              double* loss, double* dX, double* grad) {
    if (h && h->B > 1) return ACAC_E_ARG;
    if (!h || !X || !target || !dX) return ACAC_E_ARG;
    Join join(h);
    try {
        double gl[4];
        const int st = loss_and_grad(h, X, target, w_energy, w_misfit, loss, dX, gl);
        if (grad)
            for (int i = 0; i < 4; ++i) grad[i] = gl[i];
        return st;
    } catch (Err e) {
        return e.code;
    }
}

int acac_adjoint_step(acac_handle* h, const double* X1, const double* X0, double dt, const double* lam1,
                      double* lam0, double* grad, double rtol, int* gmres_its) {
    if (h && (h->B > 1 || h->mixed || h->p.subdomain_solver != ACAC_SUB_ILU0)) return ACAC_E_ARG;
    if (!h || !X1 || !X0 || !lam1 || !lam0 || !(dt > 0) || !(rtol > 0)) return ACAC_E_ARG;
    Join join(h);
    try {
        adjoint_buffers(h);
        double gl[4] = {0.0, 0.0, 0.0, 0.0};
        int its = 0;
        const int st = adjoint_step(h, X1, X0, dt, lam1, lam0, gl, rtol, &its);
        CU(cudaStreamSynchronize(h->stream));
        if (grad)
            for (int i = 0; i < 4; ++i) grad[i] = gl[i];
        if (gmres_its) *gmres_its = its;
        return st;
    } catch (Err e) {
        return e.code;
    }
}

int acac_adjoint(acac_handle* h, const double* u0, const double* v0, int nsteps, double dt, int checkpoint_every,
                 const double* u_target, const double* v_target, double w_energy, double w_misfit, double rtol,
                 double* loss, double* du0, double* dv0, double* grad, int* gmres_its) {
    if (h && (h->B > 1 || h->mixed || h->p.subdomain_solver != ACAC_SUB_ILU0)) return ACAC_E_ARG;
    if (!h || !u0 || !v0 || !u_target || !v_target || !du0 || !dv0 || nsteps < 1 || !(dt > 0) ||
        checkpoint_every < 1 || !(rtol > 0))
        return ACAC_E_ARG;
    Join join(h);
    const size_t N = h->N, n2 = 2 * N;
    const int every = std::min(checkpoint_every, nsteps);
    const int nckpt = (nsteps + every - 1) / every;
    double* store = nullptr;   // nckpt checkpoints and U^K, then every + 1 states of one segment
    struct Free {
        double** p;
        ~Free() {
            if (*p) cudaFree(*p);
        }
    } free_store{&store};
    try {
        adjoint_buffers(h);
        dmalloc(&store, 8 * n2 * (size_t)(nckpt + 1 + every + 1));
        double* seg = store + n2 * (nckpt + 1);
        double* lam = h->adj + n2;
        double* tgt = h->adj + 3 * n2;
        CU(cudaMemcpyAsync(tgt, u_target, N * 8, cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaMemcpyAsync(tgt + N, v_target, N * 8, cudaMemcpyDeviceToDevice, h->stream));
        // forward, keeping every `every`-th state
        CU(cudaMemcpyAsync(h->X0, u0, N * 8, cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaMemcpyAsync(h->X0 + N, v0, N * 8, cudaMemcpyDeviceToDevice, h->stream));
        int its = 0;
        auto step_from_X0 = [&](acac_step_info* info) {
            memset(info, 0, sizeof(*info));
            set_dt0(h, dt);
            std::vector<int> sv;
            nks_dispatch(h, std::vector<int>(1, 1), sv, info);
            return sv[0];
        };
        for (int k = 0; k < nsteps; ++k) {
            if (k % every == 0)
                CU(cudaMemcpyAsync(store + n2 * (k / every), h->X0, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
            acac_step_info info;
            const int st = step_from_X0(&info);
            if (st != ACAC_OK) return st;
            CU(cudaMemcpyAsync(h->X0, h->X, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
        }
        CU(cudaMemcpyAsync(store + n2 * nckpt, h->X0, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
        double g[4];
        int st = loss_and_grad(h, h->X0, tgt, w_energy, w_misfit, loss, lam, g);
        if (st != ACAC_OK) return st;
        // backward, one segment at a time from its checkpoint
        for (int c = nckpt - 1; c >= 0; --c) {
            const int k0 = c * every, k1 = std::min(k0 + every, nsteps);
            CU(cudaMemcpyAsync(seg, store + n2 * c, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
            CU(cudaMemcpyAsync(h->X0, seg, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
            for (int k = k0; k < k1 - 1; ++k) {
                acac_step_info info;
                st = step_from_X0(&info);
                if (st != ACAC_OK) return st;
                CU(cudaMemcpyAsync(seg + n2 * (k + 1 - k0), h->X, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
                CU(cudaMemcpyAsync(h->X0, h->X, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
            }
            // the segment ends at the next checkpoint (U^K for the last segment)
            CU(cudaMemcpyAsync(seg + n2 * (k1 - k0), store + n2 * (c + 1), n2 * 8, cudaMemcpyDeviceToDevice,
                               h->stream));
            for (int k = k1 - 1; k >= k0; --k) {
                st = adjoint_step(h, seg + n2 * (k + 1 - k0), seg + n2 * (k - k0), dt, lam, lam, g, rtol, &its);
                if (st != ACAC_OK) return st;
            }
        }
        CU(cudaMemcpyAsync(du0, lam, N * 8, cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaMemcpyAsync(dv0, lam + N, N * 8, cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        if (grad)
            for (int i = 0; i < 4; ++i) grad[i] = g[i];
        if (gmres_its) *gmres_its = its;
        return ACAC_OK;
    } catch (Err e) {
        return e.code;
    }
}

int acac_autotune(const acac_params* p, const double* u, const double* v, int trial_steps, void* cuda_stream,
                  acac_params* best, double* best_ms_per_step, int* ncandidates) {
    if (!p || !u || !v || !best || trial_steps < 1) return ACAC_E_ARG;
    int st = validate_params(p);
    if (st != ACAC_OK) return st;
    const int dim = p->dim;
    const size_t N = (size_t)p->n[0] * p->n[1] * (dim == 3 ? p->n[2] : 1) * p->batch;   // all members
    // candidates: the given partition, and near-cubic boxes of owned width W in every
    // direction for W in a ladder, each with overlap 1 and 2
    std::vector<acac_params> cand;
    auto add = [&](const acac_params& q) {
        if (validate_params(&q) != ACAC_OK) return;
        for (const acac_params& c : cand)
            if (c.ras_overlap == q.ras_overlap && c.ras_parts[0] == q.ras_parts[0] &&
                c.ras_parts[1] == q.ras_parts[1] && (dim == 2 || c.ras_parts[2] == q.ras_parts[2]))
                return;
        for (int a = 0; a < dim; ++a) {
            const int w = (p->n[a] + q.ras_parts[a] - 1) / q.ras_parts[a] + 2 * q.ras_overlap;
            if (w < 4 || w > 250 || (p->bc == ACAC_BC_PERIODIC && w > p->n[a] - 2)) return;
        }
        cand.push_back(q);
    };
    add(*p);
    const int ladder[] = {12, 16, 24, 32, 48, 64, 96, 128, 192, 240};
    for (int W : ladder)
        for (int d = 1; d <= 2; ++d) {
            acac_params q = *p;
            q.ras_overlap = d;
            for (int a = 0; a < dim; ++a) q.ras_parts[a] = std::max(1, (p->n[a] + W - 1) / W);
            add(q);
        }
    if (ncandidates) *ncandidates = (int)cand.size();
    double* X = nullptr;
    if (cudaMalloc((void**)&X, 2 * N * sizeof(double)) != cudaSuccess) return ACAC_E_NOMEM;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double best_ms = -1.0;
    int rc = ACAC_E_DIVERGED;   // when no candidate completes its trial steps
    for (const acac_params& q : cand) {
        acac_handle* h = nullptr;
        if (acac_create(&q, cuda_stream, &h) != ACAC_OK) continue;
        // one untimed step from (u, v) (first-use costs: shared-memory limits, graph
        // capture), then trial_steps timed steps continuing from it: every candidate
        // follows the same trajectory
        bool ok = cudaMemcpyAsync(X, u, N * 8, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
                  cudaMemcpyAsync(X + N, v, N * 8, cudaMemcpyDeviceToDevice, s) == cudaSuccess &&
                  acac_step(h, X, X + N, nullptr) == ACAC_OK && cudaStreamSynchronize(s) == cudaSuccess;
        double ms = -1.0;
        if (ok) {
            const auto t0 = std::chrono::steady_clock::now();
            for (int k = 0; ok && k < trial_steps; ++k) ok = acac_step(h, X, X + N, nullptr) == ACAC_OK;
            ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
            ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() /
                 trial_steps;
        }
        acac_destroy(h);
        if (ok && (best_ms < 0 || ms < best_ms)) {
            best_ms = ms;
            *best = q;
            rc = ACAC_OK;
        }
    }
    cudaFree(X);
    if (best_ms_per_step) *best_ms_per_step = best_ms;
    return rc;
}

int acac_energy(acac_handle* h, const double* u, const double* v, double* energy, double* mass) {
    if (!h || !u || !v) return ACAC_E_ARG;
    Join join(h);
    try {
        const size_t N = h->N;
        // member states [u | v] in tmpd, then one launch over the members
        KLA(ACAC_K_VECTOR, 32.0 * N, 0.0, launch_pack_members(u, v, h->tmpd, (long long)N, 1, h->stream, all_members(h)));
        std::vector<double> e, ms;
        std::vector<int> bad;
        energy_members(h, -1, h->tmpd, e, ms, bad);
        int st = ACAC_OK;
        for (int m = 0; m < h->B; ++m) {
            if (energy) energy[m] = e[m];
            if (mass) mass[m] = ms[m];
            if (bad[m] && st == ACAC_OK) st = ACAC_E_DOMAIN;
        }
        return st;
    } catch (Err e) {
        return e.code;
    }
}

int acac_step(acac_handle* h, double* u, double* v, acac_step_info* info) {
    if (!h || !u || !v) return ACAC_E_ARG;
    Join join(h);
    try {
        return step_members(h, u, v, info);
    } catch (Err e) {
        if (info)
            for (int m = 0; m < h->B; ++m) info[m].status = e.code;
        return e.code;
    }
}

int acac_step_host(acac_handle* h, double* u_host, double* v_host, acac_step_info* info) {
    if (!h || !u_host || !v_host) return ACAC_E_ARG;
    Join join(h);
    try {
        const size_t N = h->N * h->B;
        CU(cudaMemcpyAsync(h->stage, u_host, N * 8, cudaMemcpyHostToDevice, h->stream));
        CU(cudaMemcpyAsync(h->stage + N, v_host, N * 8, cudaMemcpyHostToDevice, h->stream));
        int st;
        try {
            st = step_members(h, h->stage, h->stage + N, info);
        } catch (Err e) {
            if (info)
                for (int m = 0; m < h->B; ++m) info[m].status = e.code;
            st = e.code;
        }
        // every member is copied back: a failed member's fields are unchanged
        CU(cudaMemcpyAsync(u_host, h->stage, N * 8, cudaMemcpyDeviceToHost, h->stream));
        CU(cudaMemcpyAsync(v_host, h->stage + N, N * 8, cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        return st;
    } catch (Err e) {
        return e.code;
    }
}

int acac_wait_selftest(void* stream, int mode) {
    if (mode != 0 && mode != 1) return ACAC_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return ACAC_E_NOMEM;
    int host = ACAC_E_CUDA, st = ACAC_E_CUDA;
    if (cudaMemsetAsync(d, 0, sizeof(int), s) == cudaSuccess && launch_wait_selftest(mode, d, s) == cudaSuccess &&
        cudaMemcpyAsync(&host, d, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess)
        st = host;
    cudaFree(d);
    return st;
}

int acac_subdomain_pattern(int dim, int W, int H, int D, int solver, int* ptr, int* col, long long cap,
                           long long* nnz) {
    if ((dim != 2 && dim != 3) || W < 1 || H < 1 || (dim == 3 && D < 1) || !nnz) return ACAC_E_ARG;
    if (solver != ACAC_SUB_ILU1 && solver != ACAC_SUB_ILU2 && solver != ACAC_SUB_LU) return ACAC_E_ARG;
    if ((long long)W * H * (dim == 3 ? D : 1) > 250LL * 250) return ACAC_E_ARG;
    try {
        const SparseShape S = build_sparse_shape(dim, W, H, D, solver == ACAC_SUB_LU ? -1 : solver);
        *nnz = (long long)S.col.size();
        if (!ptr || !col || cap < *nnz) return ACAC_E_ARG;
        std::copy(S.ptr.begin(), S.ptr.end(), ptr);
        std::copy(S.col.begin(), S.col.end(), col);
        return ACAC_OK;
    } catch (...) {
        return ACAC_E_NOMEM;
    }
}

}  // extern "C"
