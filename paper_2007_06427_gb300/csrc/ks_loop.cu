// ks_loop.cu - kernels and C-ABI of the KS loop tau-descent library (sm_103a).
//
// The kernels wrap the per-CTA items of ks_items.cuh: every launch runs one phase of a
// tau-step over all work items of the batch.  The host side owns the handle (device
// workspace, tables, launch shapes) and sequences the phases for the public calls declared
// in include/ks_loop.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ks_cluster.cuh"
#include "ks_items.cuh"
#include "ks_loop.h"

using namespace ks;

#define KS_VERSION_STRING "ks_loop 0.1 (sm_103a)"

// ------------------------------------------------------------------------------------------
// Kernels
// ------------------------------------------------------------------------------------------
// Per-phase launches.  Each CTA first copies the twiddles its transforms read (nm entries,
// nm = the longest transform) into a compact bank-swizzled table at tw_off, after its item
// buffers; the items read them there (the same values as the global table: the same bits).
template <typename R>
__device__ __forceinline__ Bufs<R> stage_twiddles(const Bufs<R>& p, unsigned char* smem,
                                                  int tw_off, int nm) {
    cpx<R>* tws = reinterpret_cast<cpx<R>*>(smem + tw_off);
    load_twiddles_compact(tws, p.tw, nm);
    cp_async_wait();
    __syncthreads();
    Bufs<R> q = p;
    q.tw = tws;
    q.twsh = __ffs(NMAX / nm) - 1;
    return q;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_rows(Dims d, Bufs<R> p, int nitems, int tw_off, int nm) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Bufs<R> q = stage_twiddles(p, smem, tw_off, nm);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) row_item<R, MODE, true>(d, q, it, smem);
    if constexpr (MODE == ROW_ADJ) loops_scalars(d, q, q.par, blockIdx.x, gridDim.x);
}

template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_cols(Dims d, Bufs<R> p, int nitems, int tw_off, int nm) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Bufs<R> q = stage_twiddles(p, smem, tw_off, nm);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) col_item<R, MODE, true>(d, q, it, smem, q.par);
}

// float grid -> double grid
__global__ void k_grid_f2d(const float* src, double* dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

// double band -> float band (every loop)
__global__ void k_band_d2f(const cpx<double>* src, cpx<float>* dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = mk<float>((float)src[i].x, (float)src[i].y);
}

// 2 pi / T for parity 0 after a state load
__global__ void k_prep_wT(const double* T, double* wT, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) wT[b] = 2.0 * 3.14159265358979323846 / T[b];
}

// ---- grid-wide barrier with a bounded wait -------------------------------------------------
// Sense-free generation barrier: each CTA reads the generation, arrives on the counter; the
// last arrival resets the counter and bumps the generation.  Waiters give up after about a
// second (global timer), set the error word and leave; every CTA then returns at its next
// barrier, so an inconsistent launch ends instead of hanging.
struct GridBar {
    unsigned int* count;
    unsigned int* gen;
    int* err;
    unsigned int extra;  // arrivals expected beyond the grid: 0, or 1 to test the timeout path
};

#define KS_SPIN_LIMIT (1u << 26)
#define KS_WAIT_NS 1000000000ull

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_sync(const GridBar& g) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int my = ld_acquire_gpu(g.gen);
        __threadfence();
        const unsigned int a = atomicAdd(g.count, 1u);
        int good = 1;
        if (a == gridDim.x - 1 + g.extra) {
            atomicExch(g.count, 0u);
            __threadfence();
            atomicAdd(g.gen, 1u);
        } else {
            // bounded wait: give up after KS_WAIT_NS of the GPU's global timer (or, as a
            // second guard, KS_SPIN_LIMIT polls)
            const unsigned long long t0 = globaltimer_ns();
            unsigned int it = 0;
            while (ld_acquire_gpu(g.gen) == my) {
                if (++it > KS_SPIN_LIMIT || ((it & 63) == 0 && globaltimer_ns() - t0 > KS_WAIT_NS)) {
                    atomicExch(g.err, 1);
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*(volatile int*)g.err) good = 0;
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// All phases of nsteps tau-steps in one cooperative launch: every CTA walks the row items,
// barrier, the column items, barrier, ... (four phases per step).
// The CTA's twiddles (the entries its transforms read, at bank-swizzled positions) are copied
// to shared memory at tw_off once per launch; the items then read them there instead of from
// the global table (the same values, so the same bits as the per-phase launches).
// Launch bounds: always COL_ACC_LANES = 128 threads; six resident blocks per SM caps the
// registers at 85 (80 used, no spills; with (256) alone ptxas chose 64 and spilled).
template <typename R>
__global__ void __launch_bounds__(128, 6) k_persist(Dims d, Bufs<R> p, int nsteps, int par0,
                                                 int nrow, int ncol, GridBar bar, int tw_off,
                                                 int nm) {
    extern __shared__ __align__(16) unsigned char smem[];
    cpx<R>* tws = reinterpret_cast<cpx<R>*>(smem + tw_off);
    load_twiddles(tws, p.tw, nm);
    cp_async_wait();
    __syncthreads();
    Bufs<R> q = p;
    q.tw = tws;
    // column items per phase (pairs of columns in the centre-symmetric subspace); ncol, the
    // launch's upper bound, is the count of single columns
    const int ncol_r = min(ncol, col_item_count(d, p.xi, COL_RESID));
    const int ncol_u = min(ncol, col_item_count(d, p.xi, COL_UPDATE));
    for (int s = 0; s < nsteps; ++s) {
        const int par = (par0 + s) & 1;
        for (int it = blockIdx.x; it < nrow; it += gridDim.x) row_item<R, ROW_NONLIN, true>(d, q, it, smem);
        if (!grid_sync(bar)) return;
        for (int it = blockIdx.x; it < ncol_r; it += gridDim.x) col_item<R, COL_RESID, true>(d, q, it, smem, par);
        if (!grid_sync(bar)) return;
        for (int it = blockIdx.x; it < nrow; it += gridDim.x) row_item<R, ROW_ADJ, true>(d, q, it, smem, par);
        loops_scalars(d, q, par, blockIdx.x, gridDim.x);
        if (!grid_sync(bar)) return;
        for (int it = blockIdx.x; it < ncol_u; it += gridDim.x) col_item<R, COL_UPDATE, true>(d, q, it, smem, par);
        if (s + 1 < nsteps && !grid_sync(bar)) return;
    }
}

// J = L sum_j Jpart, dJ/dT = 2 L^dag_2 = 2 (2 pi L / T^2) sum_j L2part, per loop.
// only loops with prec[b] == myprec are written when mask != 0.
template <typename P>
__global__ void k_finalize(int B, int nkx, double L, const P* Jpart, const P* L2part,
                           const double* T, const int* prec, int myprec, int mask, double* J,
                           double* dJdT, double* sqrtJ) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (mask && prec[b] != myprec) return;
    double sj = 0.0, sl = 0.0;
    for (int c = 0; c < nkx; ++c) {
        sj += widen(Jpart[(size_t)b * nkx + c]);
        sl += widen(L2part[(size_t)b * nkx + c]);
    }
    const double Tb = T[b];
    const double Jb = L * sj;
    if (J) J[b] = Jb;
    if (dJdT) dJdT[b] = 2.0 * L * 2.0 * 3.14159265358979323846 * sl / (Tb * Tb);
    if (sqrtJ) sqrtJ[b] = sqrt(Jb);
}

// float band -> double band for the loops flagged in sel[b] (mixed-precision switch).
__global__ void k_band_f2d(const cpx<float>* src, cpx<double>* dst, const long long* boff,
                           const int* sel, int B, int nkx, const int* ks) {
    const int b = blockIdx.y;
    if (b >= B || !sel[b]) return;
    const long long n = (long long)nkx * (2 * ks[b] + 1);
    const long long o = boff[b];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cpx<float> v = src[o + i];
        dst[o + i] = mk<double>((double)v.x, (double)v.y);
    }
}

// ------------------------------------------------------------------------------------------
// Error reporting
// ------------------------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

// lets the allocation-free entry point report through ks_last_error()
void ks_internal_set_error(const char* msg) { g_err = msg ? msg : ""; }

#define KS_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? KS_ERR_OOM : KS_ERR_CUDA,        \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

#define KS_TRY(expr)                \
    do {                            \
        int rc_ = (expr);           \
        if (rc_ != KS_OK) return rc_; \
    } while (0)

// ------------------------------------------------------------------------------------------
// Handle
// ------------------------------------------------------------------------------------------
namespace {

constexpr int P64 = 0, P32 = 1;

struct Work {
    void* uh[2] = {nullptr, nullptr};
    void* rh[2] = {nullptr, nullptr};
    void* gh[2] = {nullptr, nullptr};
    void* M[2] = {nullptr, nullptr};
    void* U[2] = {nullptr, nullptr};
    void* io[2] = {nullptr, nullptr};
    double* T = nullptr;       // [2][B]
    double* wT = nullptr;      // [2][B] 2 pi / T
    double* Jpart = nullptr;   // [B][nkx]
    double* L2part = nullptr;  // [B][nkx]
    int* status = nullptr;
    int* prec = nullptr;
    long long* steps = nullptr;
    double* sqrtJ = nullptr;
    double* J = nullptr;       // [B] finalize outputs
    double* dJdT = nullptr;    // [B]
    int* sel = nullptr;        // [B] selection flags (switch)
    int par = 0;
    bool mix_valid[2] = {false, false};
};

struct Launch {
    int threads = 128;
    int grid = 0;
    size_t smem = 0;    // item buffers plus the compact twiddle table
    size_t tw_off = 0;  // the item buffers' size: offset of the twiddle table
};

}  // namespace

struct ks_loop {
    int dev = 0;
    Dims d{};
    int mode = KS_FP64;
    double tol = 1e-10, switch_tol = 0.0;
    long long max_steps = 1000000;
    int chunk = 1000;
    int autotune = 0;
    long long stall_window = 40000;
    double stall_drop = 1e-3;
    std::vector<int> ns, lgns, ksv;
    std::vector<long long> boff, moff, goff;
    long long nband = 0, nmix = 0, ngrid = 0;
    int nsmax = 0;
    int rows_per_tile = 8;
    std::vector<RowItem> rows;
    std::vector<int> colorder;
    bool need[2] = {false, false};  // precisions allocated for the state workspace
    int api_prec = P64;
    // device tables
    int *d_ns = nullptr, *d_lgns = nullptr, *d_ks = nullptr, *d_colorder = nullptr;
    long long *d_boff = nullptr, *d_moff = nullptr, *d_goff = nullptr;
    RowItem* d_rows = nullptr;
    void* d_tw[2] = {nullptr, nullptr};
    void* d_qv[2] = {nullptr, nullptr};
    void* d_lin[2] = {nullptr, nullptr};
    void* d_cq[2] = {nullptr, nullptr};
    void* d_insv[2] = {nullptr, nullptr};
    // launch path of each precision (index P64, P32): 0 = cluster-resident kernel when its plan
    // fits, else 1; 1 = grid-persistent cooperative kernel; 2 = four launches per tau-step
    int path[2] = {0, 0};
    int force_cluster = 0;          // 0: choose the cluster size; else use this one
    int cexchange = 1;              // cluster kernel: mbarrier exchanges where the plan has room
    int force_mb = 0;               // cluster kernel variant: 0 by occupancy, 1 or 2 forced
    ClusterPlan cplan[3] = {};      // double, float, double + float adjoint; bytes = 0: unavailable
    int cthreads = 128;
    int cgrid[3] = {0, 0, 0};
    int finish_f32_adjoint = 0;     // mixed descents: 1 = finishing steps form the adjoint in float
    // mixed descents: probe of the float floor (knobs "switch_probe", "switch_probe_steps")
    int switch_probe = 1;
    long long probe_steps = 1000;
    int xi = 0;                     // 1: loads, gradients and updates projected onto the Xi subspace
    // ks_descend with the extrapolation of App. C (knob "extrapolate")
    int extrapolate = 0;
    double extrap_start = 1e-3;  // sqrt(J) below which a loop takes its first anchor (App. C)
    double extrap_drop = 0.5;    // extrapolate once sqrt(J) has fallen to this fraction of the anchor's
    double* anc = nullptr;          // [nband] complex double: each loop's anchor band
    double* cand = nullptr;         // [nband] complex double: the current bands, widened
    double* coef = nullptr;         // [B] extrapolation coefficient of each loop (0: none)
    int* esel = nullptr;            // [3][B] selections: new anchor, accepted, rejected
    std::vector<double> anc_sq, anc_T;  // sqrt(J) and T at each anchor (sqrt(J) < 0: no anchor)
    long long n_extrap = 0, n_extrap_rejected = 0;
    int test_barrier_extra = 0;     // test hook: the grid barrier waits for arrivals that never come
    // persistent kernel
    bool persistent = true;
    int pgrid[2] = {0, 0};
    size_t psmem[2] = {0, 0};
    int ptw_off[2] = {0, 0};  // offset of the twiddle table in the persistent kernel's smem
    unsigned int* d_bar = nullptr;  // count, gen
    int* d_err = nullptr;
    Work st;   // resident descent state
    Work api;  // scratch for ks_residual / ks_adjoint_grad
    Launch lrow[2], lcol[2];
    bool state_set = false;
    std::vector<void*> allocs;
    // profiling: per-kind event pairs around every launch when enabled
    bool prof = false;
    long long launches = 0;
    std::vector<std::string> kind_names;
    std::vector<double> kind_ms;
    std::vector<long long> kind_count;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    // a second stream for the double-precision cluster launch of a mixed batch, so that it runs
    // beside the float one (created on first use; non-blocking, ordered by the two events)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // four-launch form: runs of tau-steps captured once as CUDA graphs and replayed (knob
    // "graph"); a graph is keyed by everything its launches read from the host side
    int graph = 1;
    cudaStream_t gcap = nullptr, gcap2 = nullptr;  // capture streams (never executed on)
    cudaEvent_t gfork = nullptr, gjoin = nullptr;
    struct StepGraph {
        cudaGraphExec_t exec;
        const void* work;  // the workspace whose buffers the launches use
        bool live[2];
        double tol, swt;
        int par, xi, steps;
        long long launches;  // kernel launches in one replay
    };
    std::vector<StepGraph> graphs;
    long long graph_replays = 0;
    // convergence history recorded by ks_descend at every read-back: (steps, sqrtJ, prec)
    std::vector<std::vector<long long>> hist_steps;
    std::vector<std::vector<double>> hist_sqrtJ;
    std::vector<std::vector<int>> hist_prec;
    // host mirrors
    std::vector<int> h_status, h_prec;
    std::vector<double> h_sqrtJ;
    std::vector<long long> h_steps;
};

namespace {

int dev_alloc(ks_loop* h, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? KS_ERR_OOM : KS_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->allocs.push_back(*p);
    return KS_OK;
}

template <typename T>
int upload(ks_loop* h, T** dptr, const std::vector<T>& v) {
    void* p = nullptr;
    KS_TRY(dev_alloc(h, &p, v.size() * sizeof(T)));
    if (!v.empty()) KS_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dptr = reinterpret_cast<T*>(p);
    return KS_OK;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// exp(2 pi i t / NMAX) with octant symmetry so that the table is exactly symmetric.
void twiddles(std::vector<double>& re, std::vector<double>& im) {
    const int N = NMAX;
    re.assign(N, 0.0);
    im.assign(N, 0.0);
    const double two_pi = 6.283185307179586476925286766559;
    std::vector<double> c(N / 4 + 1), s(N / 4 + 1);
    for (int t = 0; t <= N / 8; ++t) {
        c[t] = std::cos(two_pi * t / N);
        s[t] = std::sin(two_pi * t / N);
    }
    for (int t = N / 8 + 1; t <= N / 4; ++t) {
        c[t] = s[N / 4 - t];
        s[t] = c[N / 4 - t];
    }
    for (int t = 0; t < N; ++t) {
        const int qd = t / (N / 4), r = t % (N / 4);
        double a = c[r], b = s[r];
        switch (qd) {
            case 0: re[t] = a; im[t] = b; break;
            case 1: re[t] = -b; im[t] = a; break;
            case 2: re[t] = -a; im[t] = -b; break;
            default: re[t] = b; im[t] = -a; break;
        }
    }
}

int alloc_work(ks_loop* h, Work& w, const bool* precs) {
    const int B = h->d.B;
    for (int pr = 0; pr < 2; ++pr) {
        if (!precs[pr]) continue;
        const size_t cs = pr == P64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
        const size_t rs = pr == P64 ? sizeof(double) : sizeof(float);
        KS_TRY(dev_alloc(h, &w.uh[pr], h->nband * cs));
        KS_TRY(dev_alloc(h, &w.rh[pr], h->nband * cs));
        KS_TRY(dev_alloc(h, &w.gh[pr], h->nband * cs));
        KS_TRY(dev_alloc(h, &w.M[pr], h->nmix * cs));
        KS_TRY(dev_alloc(h, &w.U[pr], h->ngrid * rs));
        KS_TRY(dev_alloc(h, &w.io[pr], h->ngrid * rs));
        KS_CUDA(cudaMemset(w.uh[pr], 0, h->nband * cs));
        KS_CUDA(cudaMemset(w.rh[pr], 0, h->nband * cs));
        KS_CUDA(cudaMemset(w.gh[pr], 0, h->nband * cs));
    }
    void* p = nullptr;
    KS_TRY(dev_alloc(h, &p, 2 * B * sizeof(double)));
    w.T = (double*)p;
    KS_TRY(dev_alloc(h, &p, 2 * B * sizeof(double)));
    w.wT = (double*)p;
    KS_TRY(dev_alloc(h, &p, (size_t)B * h->d.nkx * sizeof(double)));
    w.Jpart = (double*)p;
    KS_TRY(dev_alloc(h, &p, (size_t)B * h->d.nkx * sizeof(double)));
    w.L2part = (double*)p;
    KS_TRY(dev_alloc(h, &p, B * sizeof(int)));
    w.status = (int*)p;
    KS_TRY(dev_alloc(h, &p, B * sizeof(int)));
    w.prec = (int*)p;
    KS_TRY(dev_alloc(h, &p, B * sizeof(long long)));
    w.steps = (long long*)p;
    KS_TRY(dev_alloc(h, &p, B * sizeof(double)));
    w.sqrtJ = (double*)p;
    KS_TRY(dev_alloc(h, &p, B * sizeof(double)));
    w.J = (double*)p;
    KS_TRY(dev_alloc(h, &p, B * sizeof(double)));
    w.dJdT = (double*)p;
    KS_TRY(dev_alloc(h, &p, B * sizeof(int)));
    w.sel = (int*)p;
    KS_CUDA(cudaMemset(w.status, 0, B * sizeof(int)));
    KS_CUDA(cudaMemset(w.steps, 0, B * sizeof(long long)));
    KS_CUDA(cudaMemset(w.sqrtJ, 0, B * sizeof(double)));
    KS_CUDA(cudaMemset(w.T, 0, 2 * B * sizeof(double)));
    return KS_OK;
}

template <typename R>
Bufs<R> make_bufs(ks_loop* h, const Work& w, int pr, int check_active, double tol,
                  double switch_tol, R* io) {
    Bufs<R> p{};
    p.ns = h->d_ns;
    p.lgns = h->d_lgns;
    p.ks = h->d_ks;
    p.boff = h->d_boff;
    p.moff = h->d_moff;
    p.goff = h->d_goff;
    p.uh = (cpx<R>*)w.uh[pr];
    p.rh = (cpx<R>*)w.rh[pr];
    p.gh = (cpx<R>*)w.gh[pr];
    p.M = (cpx<R>*)w.M[pr];
    p.U = (R*)w.U[pr];
    p.io = io;
    p.T = w.T;
    p.wT = w.wT;
    p.Jpart = reinterpret_cast<typename PartT<R>::type*>(w.Jpart);
    p.L2part = reinterpret_cast<typename PartT<R>::type*>(w.L2part);
    p.status = w.status;
    p.prec = w.prec;
    p.steps = w.steps;
    p.sqrtJ = w.sqrtJ;
    p.tw = (const cpx<R>*)h->d_tw[pr];
    p.qv = (const R*)h->d_qv[pr];
    p.lin = (const R*)h->d_lin[pr];
    p.cq = (const R*)h->d_cq[pr];
    p.insv = (const R*)h->d_insv[pr];
    p.rows = h->d_rows;
    p.colorder = h->d_colorder;
    p.myprec = pr;
    p.par = w.par;
    p.tol = tol;
    p.switch_tol = switch_tol;
    p.check_active = check_active;
    p.step_scalars = check_active;  // the tau-step contexts; the gradient pass forms none
    p.xi = h->xi;
    return p;
}

const char* const kRowNames[] = {"rows_analyze", "rows_nonlin", "rows_adj", "rows_synth"};
const char* const kColNames[] = {"cols_analyze", "cols_synth_u", "cols_synth_r", "cols_synth_g",
                                 "cols_resid", "cols_update", "cols_grad"};

int kind_id(ks_loop* h, const std::string& name) {
    for (size_t i = 0; i < h->kind_names.size(); ++i)
        if (h->kind_names[i] == name) return (int)i;
    h->kind_names.push_back(name);
    h->kind_ms.push_back(0.0);
    h->kind_count.push_back(0);
    return (int)h->kind_names.size() - 1;
}

cudaEvent_t take_event(ks_loop* h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// bracket a launch with events when profiling; count it always
struct LaunchScope {
    ks_loop* h;
    cudaStream_t s;
    int kind = -1;
    cudaEvent_t a = nullptr;
    LaunchScope(ks_loop* h_, cudaStream_t s_, const std::string& name) : h(h_), s(s_) {
        if (h->prof) {
            kind = kind_id(h, name);
            a = take_event(h);
            cudaEventRecord(a, s);
        }
    }
    void done() {
        h->launches++;
        if (h->prof && a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, s);
            h->pending.push_back(ks_loop::Rec{kind, a, b});
        }
    }
};

std::string prec_suffix(int pr) { return pr == 0 ? "_f64" : "_f32"; }

template <typename R, int MODE>
int launch_rows(ks_loop* h, const Bufs<R>& p, cudaStream_t s) {
    const int pr = std::is_same<R, double>::value ? P64 : P32;
    const Launch& l = h->lrow[pr];
    const int n = (int)h->rows.size();
    LaunchScope ls(h, s, std::string(kRowNames[MODE]) + prec_suffix(pr));
    k_rows<R, MODE><<<std::min(n, l.grid), l.threads, l.smem, s>>>(h->d, p, n, (int)l.tw_off,
                                                                     std::max(h->d.nx, h->nsmax));
    KS_CUDA(cudaGetLastError());
    ls.done();
    return KS_OK;
}

template <typename R, int MODE>
int launch_cols(ks_loop* h, const Bufs<R>& p, cudaStream_t s) {
    const int pr = std::is_same<R, double>::value ? P64 : P32;
    const Launch& l = h->lcol[pr];
    const int n = col_item_count(h->d, h->xi, MODE);
    LaunchScope ls(h, s, std::string(kColNames[MODE]) + prec_suffix(pr));
    k_cols<R, MODE><<<std::min(n, l.grid), l.threads, l.smem, s>>>(h->d, p, n, (int)l.tw_off,
                                                                     std::max(h->d.nx, h->nsmax));
    KS_CUDA(cudaGetLastError());
    ls.done();
    return KS_OK;
}

template <typename R>
int set_smem_attrs(ks_loop* h) {
    const int pr = std::is_same<R, double>::value ? P64 : P32;
    const int rs = (int)h->lrow[pr].smem, cs = (int)h->lcol[pr].smem;
#define KS_ATTR(kern, bytes) \
    KS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))
    KS_ATTR((k_rows<R, ROW_ANALYZE>), rs);
    KS_ATTR((k_rows<R, ROW_NONLIN>), rs);
    KS_ATTR((k_rows<R, ROW_ADJ>), rs);
    KS_ATTR((k_rows<R, ROW_SYNTH>), rs);
    KS_ATTR((k_cols<R, COL_ANALYZE>), cs);
    KS_ATTR((k_cols<R, COL_SYNTH_U>), cs);
    KS_ATTR((k_cols<R, COL_SYNTH_R>), cs);
    KS_ATTR((k_cols<R, COL_SYNTH_G>), cs);
    KS_ATTR((k_cols<R, COL_RESID>), cs);
    KS_ATTR((k_cols<R, COL_UPDATE>), cs);
    KS_ATTR((k_cols<R, COL_GRAD>), cs);
#undef KS_ATTR
    return KS_OK;
}

// co-resident grid size and shared memory of the persistent kernel of one precision
template <typename R>
int setup_persistent(ks_loop* h) {
    const int pr = std::is_same<R, double>::value ? P64 : P32;
    // the items' buffers, then the twiddle table (NMAX entries, swizzled positions)
    const size_t items_sm = std::max(h->lrow[pr].tw_off, h->lcol[pr].tw_off);  // 16-aligned
    const size_t sm = items_sm + (size_t)NMAX * sizeof(cpx<R>);
    h->ptw_off[pr] = (int)items_sm;
    KS_CUDA(cudaFuncSetAttribute(k_persist<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int per_sm = 0, sms = 0, coop = 0;
    KS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist<R>, COL_ACC_LANES, sm));
    KS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
    KS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->dev));
    const int items = std::max((int)h->rows.size(), h->d.B * h->d.nkx);
    h->psmem[pr] = sm;
    h->pgrid[pr] = (coop && per_sm > 0) ? std::min(items, per_sm * sms) : 0;
    return KS_OK;
}

// Shared-memory plan of the cluster kernel for cluster size C (bytes = 0 if it cannot fit).
template <typename R, typename RA>
ClusterPlan make_cluster_plan(const ks_loop* h, int C, int u_global, int smem_limit, int smem_sm,
                              int sms) {
    ClusterPlan cp{};
    const size_t cs = sizeof(cpx<R>), rs = sizeof(R);
    const int nx = h->d.nx, nkx = h->d.nkx;
    cp.C = C;
    // columns per rank: single columns, or pairs of columns in the centre-symmetric subspace
    // (the knob can change after the plan is made, so the plan holds either)
    const int npr = (h->d.kx + 1) / 2;
    cp.ncmax = std::max((nkx + C - 1) / C, 2 * ((npr + C - 1) / C));
    cp.nsmax = h->nsmax;
    cp.nkmax = 2 * (h->nsmax / 3) + 1;
    int nsmin = h->nsmax;
    for (int v : h->ns) nsmin = std::min(nsmin, v);
    cp.rmax = 0;
    for (int v : h->ns) cp.rmax = std::max(cp.rmax, cluster_rows_per_rank(v, C));
    int rt = 2;
    while (rt * 2 <= std::min(cp.rmax, 16) && 2 * (size_t)(rt * 2) * nx * cs <= 32 * 1024) rt *= 2;
    cp.rt = rt;
    cp.u_global = u_global;
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    size_t off = 0;
    cp.off_M = (int)off;
    off += al((size_t)cp.ncmax * cp.nsmax * cs);
    cp.off_uh = (int)off;
    off += al((size_t)cp.ncmax * cp.nkmax * cs);
    cp.off_rh = (int)off;
    off += al((size_t)cp.ncmax * cp.nkmax * cs);
    cp.off_U = (int)off;
    if (!u_global) off += al((size_t)cp.rmax * nx * rs);
    cp.off_scr = (int)off;
    off += al(std::max((size_t)cp.ncmax * cp.nsmax, (size_t)2 * rt * nx) * cs);
    cp.off_part = (int)off;
    off += al((size_t)2 * nkx * sizeof(double));
    cp.off_red = (int)off;
    off += al((size_t)COL_RED_DOUBLES * sizeof(double));
    cp.off_tw = (int)off;
    off += al((size_t)NMAX * cs);
    cp.off_rin = (int)off;
    off += al((size_t)nkx * cp.rmax * cs);
    cp.off_tw_a = (int)off;
    if (sizeof(RA) != sizeof(R)) off += al((size_t)NMAX * sizeof(cpx<RA>));
    cp.off_tab = (int)off;
    off += al((size_t)nkx * (3 * rs + sizeof(RA)));
    // mbarrier exchanges: a second column buffer and four mbarriers, where they fit and keep the
    // CTAs per SM that the batch's clusters can use (1 KB of each CTA's shared memory is the
    // system's).  Not for clusters of one CTA, whose cluster barrier is a block barrier (a
    // batch of 256 64x64 loops measured 2 % slower with the exchanges).
    cp.ax = 0;
    cp.off_M2 = cp.off_M;
    cp.off_bar = 0;
    if (h->cexchange && C > 1) {
        const size_t m2 = al((size_t)cp.ncmax * cp.nsmax * cs), with = off + m2 + 32;
        const size_t need = ((size_t)h->d.B * C + sms - 1) / sms;  // CTAs per SM for one wave
        const size_t per0 = (size_t)smem_sm / (off + 1024), per1 = (size_t)smem_sm / (with + 1024);
        if (with <= (size_t)smem_limit && per1 >= std::min(per0, need)) {
            cp.off_M2 = (int)off;
            cp.off_bar = (int)(off + m2);
            cp.ax = 1;
            off = with;
        }
    }
    cp.bytes = (off <= (size_t)smem_limit) ? (int)off : 0;
    return cp;
}

// Threads per CTA of the cluster kernel in plan slot `slot` (0 double, 1 float, 2 double state
// with a float adjoint) for plan cp.  At the default width of 128 threads the kernel runs one more
// warp, which forms the scalars of each step (J, the next T and 2 pi / T, the freeze decision)
// beside the four work warps: in phase B' for a double state (before, the s-transform of w_hat
// ran on three warps, two rounds of its 128 butterflies a pass), in phase A' for a float state
// (before, the scalars held up phase B': 3.7 k of 22.7 k clocks of the 64x128 float step).  The
// element loops keep to the four work warps (see k_cluster).  A double transform spread over
// five warps could put two warps on one SM sub-partition, so the double plans take the extra
// warp only when none of their transforms has more than 128 butterflies a pass; the float
// transforms are warp-owned, where a fifth warp never adds a round.
int cluster_block(const ks_loop* h, int slot, const ClusterPlan& cp) {
    if (h->cthreads != 128) return h->cthreads;
    if (slot == 1) return 160;  // float: warp-owned transforms, never more rounds with 5 warps
    const int nx = h->d.nx;
    const int lgnx = ilog2(nx);
    const int zb = cp.rt * ((lgnx & 1) ? nx / 2 : nx / 4);  // transform of u + i u_x, one per row
    const int pb = (cp.rt / 2) * (nx / 2);                   // row pairs
    const int cb = cp.ncmax * (cp.nsmax / 2);                // columns (or column pairs)
    return (zb <= 128 && pb <= 128 && cb <= 128) ? 160 : 128;
}

// the cluster kernel of a column scheme and launch-bound variant (see k_cluster)
template <typename R, typename RA>
using ClusterFn = void (*)(Dims, Bufs<R>, AdjTables<RA>, ClusterPlan, int, int, int);
template <typename R, typename RA>
ClusterFn<R, RA> cluster_fn(bool xi, int mb) {
    if (mb == 2) return xi ? k_cluster<R, RA, true, 2> : k_cluster<R, RA, false, 2>;
    return xi ? k_cluster<R, RA, true, 1> : k_cluster<R, RA, false, 1>;
}

// pick the cluster size: enough CTAs to cover the GPU (about two per SM), at most 16, and a
// plan that fits shared memory (grid rows of u in global memory if needed).  Of the kernel's
// two launch-bound variants the plan takes the one without a register cap unless the capped one
// keeps more of the batch's clusters resident at once.
// plan slots: 0 double, 1 float, 2 double state with a float adjoint (mixed finishing)
template <typename R, typename RA>
int setup_cluster(ks_loop* h) {
    const int pr = std::is_same<R, double>::value ? (std::is_same<RA, double>::value ? 0 : 2) : 1;
    h->cplan[pr] = ClusterPlan{};
    int limit = 0, sms = 0, smem_sm = 0;
    KS_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev));
    KS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev));
    KS_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->dev));
    int target = 16;
    while (target > 1 && (long long)target * h->d.B > 2LL * sms) target >>= 1;
    for (int v = 0; v < 4; ++v)
        KS_CUDA(cudaFuncSetAttribute(cluster_fn<R, RA>(v & 1, 1 + (v >> 1)),
                                     cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    // candidate sizes: powers of two from the target down.  (A size that only balances the
    // columns, e.g. 11 ranks of 2 columns for 22, gives each rank 12 rows in two x-batches and
    // measured slower than 16 ranks with one row batch each.)
    std::vector<int> cands;
    if (h->force_cluster) {
        cands.push_back(h->force_cluster);
    } else {
        for (int t = target; t >= 1; t >>= 1) cands.push_back(t);
    }
    for (int C : cands) {
        for (int ug = 0; ug < 2; ++ug) {
            ClusterPlan cp = make_cluster_plan<R, RA>(h, C, ug, limit, smem_sm, sms);
            if (!cp.bytes) continue;
            for (int v = 0; v < 4; ++v)
                KS_CUDA(cudaFuncSetAttribute(cluster_fn<R, RA>(v & 1, 1 + (v >> 1)),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, cp.bytes));
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(cluster_block(h, pr, cp));
            cfg.dynamicSmemBytes = cp.bytes;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            // resident clusters of each launch-bound variant (the fewer of its two column schemes)
            int nv[2] = {0, 0};
            for (int m = 0; m < 2; ++m) {
                nv[m] = 1 << 30;
                for (int x = 0; x < 2; ++x) {
                    int n = 0;
                    if (cudaOccupancyMaxActiveClusters(&n, cluster_fn<R, RA>(x, 1 + m), &cfg) != cudaSuccess) {
                        cudaGetLastError();
                        n = 0;
                    }
                    nv[m] = std::min(nv[m], n);
                }
            }
            cp.mb = h->force_mb ? h->force_mb : ((nv[0] >= std::min(h->d.B, nv[1])) ? 1 : 2);
            const int ncl = nv[cp.mb - 1];
            if (ncl <= 0) continue;
            h->cplan[pr] = cp;
            h->cgrid[pr] = C * std::min(h->d.B, ncl);
            return KS_OK;
        }
    }
    return KS_OK;
}

// Default launch form of each precision's steps (the "path" knob, set per precision), from
// steady-state step times on GB300 of the cluster-resident kernel against the four-launch form
// replayed as graphs, over loops of 32x64 to 256x1024 points in batches of 1-128 (and ragged
// batches of 64-1024 loops).  All forms compute the same bits, so this only sets the speed.
// P = Nx * max Ns, the points of the longest loop:
//   * ragged batches (loops of unequal Ns) of 64 or more loops: four launches per step.  One
//     cluster per loop leaves the SMs that hold the long loops working while the rest idle;
//   * double: four launches once P >= 16384, or P >= 8192 in batches of 8 or more, or when the
//     cluster plan has 1 or 2 CTAs per loop on P >= 4096 in a batch.  A double loop of that size
//     keeps each CTA of its cluster busy for long serial transforms (64x256 single loop: 54 us
//     per step resident, 38 us in four launches; 256x256: 192 against 45);
//   * float: four launches once P >= 32768, or P >= 16384 in batches of 64 or more (float
//     transforms are short enough that the resident kernel's saved launches and round trips to
//     memory win up to there: 64x256 x 32 loops 29.7 against 30.4 us; 256x1024 x 8 loops 305
//     against 83);
//   * otherwise the cluster-resident kernel.
// ks_autotune replaces the choice of the handle's bulk precision by timing.
int default_path(const ks_loop* h, int pr) {
    const int B = h->d.B;
    bool ragged = false;
    for (int b = 1; b < B; ++b) ragged |= (h->ns[b] != h->ns[0]);
    if (ragged && B >= 64) return 2;
    const long long P = (long long)h->d.nx * h->nsmax;
    if (pr == P64) {
        if (P >= 16384 || (P >= 8192 && B >= 8)) return 2;
        const int C = h->cplan[0].bytes ? h->cplan[0].C : 0;
        if (B > 1 && (C == 1 || C == 2) && P >= 4096) return 2;
        return 0;
    }
    return (P >= 32768 || (P >= 16384 && B >= 64)) ? 2 : 0;
}

// the launch form precision pr's steps take: 0 cluster-resident (where its plan fits), 1
// grid-persistent (where its cooperative grid fits), 2 four launches per step
int form_of(const ks_loop* h, int pr) {
    const int p = h->path[pr];
    if (p == 0 && h->cplan[pr].bytes > 0) return 0;
    if (p <= 1 && h->pgrid[pr] > 0) return 1;
    return 2;
}

// nsteps tau-steps of the live loops of precision pr, one cluster per loop
template <typename R, typename RA>
int run_cluster(ks_loop* h, Work& w, int pr, long long nsteps, double tol, double switch_tol,
                cudaStream_t s, bool concurrent = false) {
    Bufs<R> p = make_bufs<R>(h, w, pr, 1, tol, switch_tol, (R*)nullptr);
    p.own_frozen_only = concurrent ? 1 : 0;
    const int slot = std::is_same<R, RA>::value ? pr : 2;
    const int pa = std::is_same<RA, double>::value ? P64 : P32;
    AdjTables<RA> ta{(const cpx<RA>*)h->d_tw[pa], (const RA*)h->d_qv[pa], (const RA*)h->d_lin[pa]};
    ClusterPlan cp = h->cplan[slot];
    cp.err = h->d_err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->cgrid[slot]);
    cfg.blockDim = dim3(cluster_block(h, slot, cp));
    cfg.dynamicSmemBytes = cp.bytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cp.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    LaunchScope ls(h, s, std::string("cluster") + prec_suffix(pr) + (slot == 2 ? "_adj_f32" : ""));
    KS_CUDA(cudaLaunchKernelEx(&cfg, cluster_fn<R, RA>(h->xi != 0, cp.mb), h->d, p,
                               ta, cp, (int)nsteps, w.par,
                               w.mix_valid[pr] ? 1 : 0));
    ls.done();
    w.mix_valid[pr] = true;
    return KS_OK;
}

// nsteps tau-steps of the live loops of precision pr in one cooperative launch
template <typename R>
int run_persist(ks_loop* h, Work& w, int pr, long long nsteps, double tol, double switch_tol,
                cudaStream_t s) {
    Bufs<R> p = make_bufs<R>(h, w, pr, 1, tol, switch_tol, (R*)nullptr);
    Dims d = h->d;
    int ns_i = (int)nsteps;
    int par0 = w.par;
    int nrow = (int)h->rows.size();
    int ncol = h->d.B * h->d.nkx;
    GridBar bar{h->d_bar, h->d_bar + 1, h->d_err, (unsigned int)h->test_barrier_extra};
    int tw_off = h->ptw_off[pr];
    int nm = std::max(h->d.nx, h->nsmax);  // longest transform
    void* args[] = {&d, &p, &ns_i, &par0, &nrow, &ncol, &bar, &tw_off, &nm};
    LaunchScope ls(h, s, std::string("persist") + prec_suffix(pr));
    KS_CUDA(cudaLaunchCooperativeKernel((const void*)k_persist<R>, dim3(h->pgrid[pr]), dim3(COL_ACC_LANES),
                                        args, h->psmem[pr], s));
    ls.done();
    return KS_OK;
}

// grid -> band (u_hat) for every loop, from io
template <typename R>
int run_analyze(ks_loop* h, Work& w, int pr, R* io, cudaStream_t s) {
    Bufs<R> p = make_bufs<R>(h, w, pr, 0, 0.0, 0.0, io);
    KS_TRY((launch_rows<R, ROW_ANALYZE>(h, p, s)));
    KS_TRY((launch_cols<R, COL_ANALYZE>(h, p, s)));
    w.mix_valid[pr] = false;
    return KS_OK;
}

// band (u_hat / r_hat / G_hat) -> grid io, every loop
template <typename R, int CMODE>
int run_synth(ks_loop* h, Work& w, int pr, R* io, cudaStream_t s) {
    Bufs<R> p = make_bufs<R>(h, w, pr, 0, 0.0, 0.0, io);
    KS_TRY((launch_cols<R, CMODE>(h, p, s)));
    KS_TRY((launch_rows<R, ROW_SYNTH>(h, p, s)));
    w.mix_valid[pr] = false;
    return KS_OK;
}

// M = s-inverse of u_hat (the input of ROW_NONLIN)
template <typename R>
int run_prime(ks_loop* h, Work& w, int pr, cudaStream_t s) {
    Bufs<R> p = make_bufs<R>(h, w, pr, 0, 0.0, 0.0, (R*)nullptr);
    KS_TRY((launch_cols<R, COL_SYNTH_U>(h, p, s)));
    w.mix_valid[pr] = true;
    return KS_OK;
}

// one tau-step of every live loop of precision pr (M must hold s-inverse of u_hat)
template <typename R>
int run_step(ks_loop* h, Work& w, int pr, double tol, double switch_tol, cudaStream_t s) {
    Bufs<R> p = make_bufs<R>(h, w, pr, 1, tol, switch_tol, (R*)nullptr);
    KS_TRY((launch_rows<R, ROW_NONLIN>(h, p, s)));
    KS_TRY((launch_cols<R, COL_RESID>(h, p, s)));
    KS_TRY((launch_rows<R, ROW_ADJ>(h, p, s)));
    KS_TRY((launch_cols<R, COL_UPDATE>(h, p, s)));
    return KS_OK;
}

// residual pass (no update): J partials and r_hat for every loop of the workspace
template <typename R>
int run_residual(ks_loop* h, Work& w, int pr, cudaStream_t s) {
    Bufs<R> p = make_bufs<R>(h, w, pr, 0, 0.0, 0.0, (R*)nullptr);
    KS_TRY((launch_cols<R, COL_SYNTH_U>(h, p, s)));
    KS_TRY((launch_rows<R, ROW_NONLIN>(h, p, s)));
    KS_TRY((launch_cols<R, COL_RESID>(h, p, s)));
    w.mix_valid[pr] = false;
    return KS_OK;
}

template <typename R>
int run_gradient(ks_loop* h, Work& w, int pr, cudaStream_t s) {
    KS_TRY(run_residual<R>(h, w, pr, s));
    Bufs<R> p = make_bufs<R>(h, w, pr, 0, 0.0, 0.0, (R*)nullptr);
    KS_TRY((launch_rows<R, ROW_ADJ>(h, p, s)));
    KS_TRY((launch_cols<R, COL_GRAD>(h, p, s)));
    return KS_OK;
}

int run_finalize(ks_loop* h, Work& w, const double* T, int myprec, int mask,
                 cudaStream_t s) {
    const int B = h->d.B;
    LaunchScope ls(h, s, "finalize");
    if (myprec == P64)
        k_finalize<double><<<(B + 127) / 128, 128, 0, s>>>(B, h->d.nkx, h->d.L, w.Jpart, w.L2part, T,
                                                            w.prec, myprec, mask, w.J, w.dJdT, w.sqrtJ);
    else
        k_finalize<ff><<<(B + 127) / 128, 128, 0, s>>>(B, h->d.nkx, h->d.L, (const ff*)w.Jpart,
                                                        (const ff*)w.L2part, T, w.prec, myprec, mask,
                                                        w.J, w.dJdT, w.sqrtJ);
    KS_CUDA(cudaGetLastError());
    ls.done();
    return KS_OK;
}

// ---- pointer staging ----
bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return KS_OK;
    KS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    return KS_OK;
}

size_t elem_size(int pr) { return pr == P64 ? sizeof(double) : sizeof(float); }

int check_handle(ks_loop* h) {
    if (!h) return fail(KS_ERR_ARG, "null handle");
    KS_CUDA(cudaSetDevice(h->dev));
    return KS_OK;
}

// load [P u; T] into workspace w in precision pr (io holds u already when io_loaded)
// The projection onto the band always runs in double: a float field is widened first and the
// projected band is rounded to float afterwards, so the band of a float handle carries only
// the rounding of its coefficients, not the transform noise of a float analysis.
int load_state(ks_loop* h, Work& w, int pr, const void* u, const double* T, cudaStream_t s) {
    const size_t gb = (size_t)h->ngrid * elem_size(pr);
    void* io = w.io[pr];
    if (is_device_ptr(u)) {
        io = const_cast<void*>(u);
    } else {
        KS_TRY(copy_in(io, u, gb, s));
    }
    KS_TRY(copy_in(w.T, T, h->d.B * sizeof(double), s));
    w.par = 0;
    k_prep_wT<<<(h->d.B + 127) / 128, 128, 0, s>>>(w.T, w.wT, h->d.B);
    KS_CUDA(cudaGetLastError());
    if (pr == P64) {
        KS_TRY(run_analyze<double>(h, w, P64, (double*)io, s));
    } else {
        const long long n = h->ngrid;
        const int g = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
        k_grid_f2d<<<g, 256, 0, s>>>((const float*)io, (double*)w.io[P64], n);
        KS_CUDA(cudaGetLastError());
        KS_TRY(run_analyze<double>(h, w, P64, (double*)w.io[P64], s));
        const long long nb = h->nband;
        k_band_d2f<<<(int)std::max<long long>(1, std::min<long long>((nb + 255) / 256, 152 * 8)), 256, 0, s>>>(
            (const cpx<double>*)w.uh[P64], (cpx<float>*)w.uh[P32], nb);
        KS_CUDA(cudaGetLastError());
        w.mix_valid[P32] = false;
    }
    return KS_OK;
}

// copy a device result buffer to the caller's pointer (device or host)
int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (!dst || bytes == 0) return KS_OK;
    KS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    return KS_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Public API
// ------------------------------------------------------------------------------------------
extern "C" const char* ks_last_error(void) { return g_err.c_str(); }
extern "C" const char* ks_version(void) { return KS_VERSION_STRING; }
extern "C" unsigned long long ks_config_sizeof(void) { return sizeof(ks_config); }

int ks_autotune_impl(ks_loop* h);

extern "C" int ks_loop_create(const ks_config* cfg, ks_loop_t* out) {
    g_err.clear();
    if (!cfg || !out) return fail(KS_ERR_ARG, "null cfg or out");
    *out = nullptr;
    if (!(cfg->L > 0.0) || !std::isfinite(cfg->L)) return fail(KS_ERR_ARG, "L must be > 0");
    if (!is_pow2(cfg->nx) || cfg->nx < 8 || cfg->nx > NMAX)
        return fail(KS_ERR_ARG, "nx must be a power of two in [8, 1024]");
    if (cfg->batch < 1 || !cfg->ns) return fail(KS_ERR_ARG, "batch must be >= 1 with ns given");
    if (cfg->mode < KS_FP64 || cfg->mode > KS_MIXED) return fail(KS_ERR_ARG, "bad mode");
    if (cfg->scheme != KS_EXPLICIT && cfg->scheme != KS_IMEX) return fail(KS_ERR_ARG, "bad scheme");
    if (!(cfg->dtau > 0.0) || !std::isfinite(cfg->dtau)) return fail(KS_ERR_ARG, "dtau must be > 0");
    if (cfg->chunk < 0) return fail(KS_ERR_ARG, "chunk must be >= 0");
    for (int b = 0; b < cfg->batch; ++b)
        if (!is_pow2(cfg->ns[b]) || cfg->ns[b] < 8 || cfg->ns[b] > NMAX)
            return fail(KS_ERR_ARG, "every ns must be a power of two in [8, 1024]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(KS_ERR_CUDA, "no CUDA device");
    }

    ks_loop* h = new ks_loop();
    cudaGetDevice(&h->dev);
    const int B = cfg->batch;
    h->d.B = B;
    h->d.nx = cfg->nx;
    h->d.lgnx = ilog2(cfg->nx);
    h->d.kx = cfg->nx / 3;
    h->d.nkx = h->d.kx + 1;
    h->d.L = cfg->L;
    h->d.dtau = cfg->dtau;
    h->d.scheme = cfg->scheme;
    h->d.hx = 0.5 / (double)cfg->nx;
    h->mode = cfg->mode;
    h->tol = cfg->tol;
    h->switch_tol = cfg->switch_tol;
    h->max_steps = cfg->max_steps;
    h->chunk = cfg->chunk > 0 ? cfg->chunk : 1000;
    h->autotune = cfg->autotune;
    h->ns.resize(B);
    h->lgns.resize(B);
    h->ksv.resize(B);
    h->boff.resize(B);
    h->moff.resize(B);
    h->goff.resize(B);
    long long bo = 0, mo = 0, go = 0;
    for (int b = 0; b < B; ++b) {
        const int n = cfg->ns[b];
        h->ns[b] = n;
        h->lgns[b] = ilog2(n);
        h->ksv[b] = n / 3;
        h->boff[b] = bo;
        h->moff[b] = mo;
        h->goff[b] = go;
        bo += (long long)h->d.nkx * (2 * (n / 3) + 1);
        mo += (long long)h->d.nkx * n;
        go += (long long)n * cfg->nx;
        h->nsmax = std::max(h->nsmax, n);
    }
    h->nband = bo;
    h->nmix = mo;
    h->ngrid = go;
    // row tiles: rows_per_tile rows of one loop (even power of two, divides Ns).  Two double
    // tile buffers of rows_per_tile x Nx complex values stay within 96 KB of shared memory, and
    // small batches get smaller tiles so that at least two row items exist per SM.
    {
        long long rows_total = go / cfg->nx;
        h->rows_per_tile = 8;
        while (h->rows_per_tile > 2 &&
               (2 * (size_t)h->rows_per_tile * cfg->nx * sizeof(cpx<double>) > 96 * 1024 ||
                rows_total / h->rows_per_tile < 2 * 152))
            h->rows_per_tile >>= 1;
    }
    for (int b = 0; b < B; ++b) {
        const int nr = std::min(h->rows_per_tile, h->ns[b]);
        for (int n0 = 0; n0 < h->ns[b]; n0 += nr) h->rows.push_back(RowItem{b, n0, nr, ilog2(nr)});
    }
    // columns: longest loops first
    h->colorder.resize(B);
    for (int b = 0; b < B; ++b) h->colorder[b] = b;
    std::stable_sort(h->colorder.begin(), h->colorder.end(),
                     [&](int a, int c) { return h->ns[a] > h->ns[c]; });
    h->need[P64] = (h->mode == KS_FP64 || h->mode == KS_MIXED);
    h->need[P32] = (h->mode == KS_FP32 || h->mode == KS_MIXED);
    h->api_prec = (h->mode == KS_FP32) ? P32 : P64;

    auto cleanup = [&](int rc) {
        ks_destroy(h);
        return rc;
    };
    int rc;
    if ((rc = upload(h, &h->d_ns, h->ns)) || (rc = upload(h, &h->d_lgns, h->lgns)) ||
        (rc = upload(h, &h->d_ks, h->ksv)) || (rc = upload(h, &h->d_boff, h->boff)) ||
        (rc = upload(h, &h->d_moff, h->moff)) || (rc = upload(h, &h->d_goff, h->goff)) ||
        (rc = upload(h, &h->d_rows, h->rows)) || (rc = upload(h, &h->d_colorder, h->colorder)))
        return cleanup(rc);
    {
        std::vector<double> re, im;
        twiddles(re, im);
        std::vector<cpx<double>> t64(NMAX);
        std::vector<cpx<float>> t32(NMAX);
        for (int t = 0; t < NMAX; ++t) {
            t64[t].x = re[t];
            t64[t].y = im[t];
            t32[t].x = (float)re[t];
            t32[t].y = (float)im[t];
        }
        // per retained x-mode: q_j, q_j^2 - q_j^4, q_j^4 (q_j^2 - 1)^2; per loop: 1 / Ns
        std::vector<double> q64(h->d.nkx), l64(h->d.nkx), c64(h->d.nkx), i64v(B);
        std::vector<float> q32(h->d.nkx), l32(h->d.nkx), c32(h->d.nkx), i32v(B);
        for (int j = 0; j < h->d.nkx; ++j) {
            const double q = 2.0 * 3.14159265358979323846 * (double)j / h->d.L;
            q64[j] = q;
            l64[j] = q * q - q * q * q * q;
            c64[j] = q * q * q * q * (q * q - 1.0) * (q * q - 1.0);
            q32[j] = (float)q64[j];
            l32[j] = (float)l64[j];
            c32[j] = (float)c64[j];
        }
        for (int b = 0; b < B; ++b) {
            i64v[b] = 1.0 / (double)h->ns[b];
            i32v[b] = (float)i64v[b];
        }
        cpx<double>* p64 = nullptr;
        cpx<float>* p32 = nullptr;
        double *qq64 = nullptr, *ll64 = nullptr, *cc64 = nullptr, *ii64 = nullptr;
        float *qq32 = nullptr, *ll32 = nullptr, *cc32 = nullptr, *ii32 = nullptr;
        if ((rc = upload(h, &p64, t64)) || (rc = upload(h, &p32, t32)) ||
            (rc = upload(h, &qq64, q64)) || (rc = upload(h, &qq32, q32)) ||
            (rc = upload(h, &ll64, l64)) || (rc = upload(h, &ll32, l32)) ||
            (rc = upload(h, &cc64, c64)) || (rc = upload(h, &cc32, c32)) ||
            (rc = upload(h, &ii64, i64v)) || (rc = upload(h, &ii32, i32v)))
            return cleanup(rc);
        h->d_tw[P64] = p64;
        h->d_tw[P32] = p32;
        h->d_qv[P64] = qq64;
        h->d_qv[P32] = qq32;
        h->d_lin[P64] = ll64;
        h->d_lin[P32] = ll32;
        h->d_cq[P64] = cc64;
        h->d_cq[P32] = cc32;
        h->d_insv[P64] = ii64;
        h->d_insv[P32] = ii32;
        void* pb = nullptr;
        if ((rc = dev_alloc(h, &pb, 4 * sizeof(unsigned int)))) return cleanup(rc);
        h->d_bar = (unsigned int*)pb;
        if ((rc = dev_alloc(h, &pb, sizeof(int)))) return cleanup(rc);
        h->d_err = (int*)pb;
        if (cudaMemset(h->d_bar, 0, 4 * sizeof(unsigned int)) != cudaSuccess ||
            cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess)
            return cleanup(fail(KS_ERR_CUDA, "barrier init failed"));
    }
    // double buffers always exist: every projection onto the band runs in double
    bool st_need[2] = {true, h->need[P32]};
    bool api_need[2] = {true, h->api_prec == P32};
    if ((rc = alloc_work(h, h->st, st_need)) || (rc = alloc_work(h, h->api, api_need)))
        return cleanup(rc);
    // launch shapes.  Block sizes from step times of the four-launch form on GB300: 256-thread
    // row items for rows of 256 points or more (256 x 1024, 8 loops: 505 against 546 us per
    // double step), 256-thread column items only when the columns are fewer than the SMs and
    // long (one 256 x 1024 loop: 102 against 113 us); batches with more column items run
    // them faster at 128 threads (ragged 64 x {32..256}, 256 loops: 405 against 479 us).
    const int ncolitems = B * h->d.nkx;
    for (int pr = 0; pr < 2; ++pr) {
        const size_t cs = pr == P64 ? sizeof(cpx<double>) : sizeof(cpx<float>);
        const size_t tw_bytes = (size_t)std::max(h->d.nx, h->nsmax) * cs;  // compact table
        Launch& lr = h->lrow[pr];
        lr.threads = h->d.nx >= 256 ? 256 : 128;
        lr.tw_off = (2 * (size_t)h->rows_per_tile * h->d.nx * cs + 15) & ~(size_t)15;
        lr.smem = lr.tw_off + tw_bytes;
        lr.grid = 152 * 16;
        Launch& lc = h->lcol[pr];
        lc.threads = (ncolitems < 152 && h->nsmax >= 256) ? 256 : 128;
        lc.tw_off = (2 * (size_t)h->nsmax * cs + COL_RED_DOUBLES * sizeof(double) + 15) & ~(size_t)15;
        lc.smem = lc.tw_off + tw_bytes;
        lc.grid = 152 * 16;
    }
    if ((rc = set_smem_attrs<double>(h)) || (rc = set_smem_attrs<float>(h))) return cleanup(rc);
    if ((rc = setup_persistent<double>(h)) || (rc = setup_persistent<float>(h))) return cleanup(rc);
    if ((rc = setup_cluster<double, double>(h)) || (rc = setup_cluster<float, float>(h)) ||
        (h->mode == KS_MIXED && (rc = setup_cluster<double, float>(h))))
        return cleanup(rc);
    h->h_status.assign(B, 0);
    h->h_prec.assign(B, 0);
    h->h_sqrtJ.assign(B, 0.0);
    h->h_steps.assign(B, 0);
    h->path[P64] = default_path(h, P64);
    h->path[P32] = default_path(h, P32);
    if (h->autotune && (rc = ks_autotune_impl(h))) return cleanup(rc);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cleanup(fail(KS_ERR_CUDA, cudaGetErrorString(e)));
    *out = h;
    return KS_OK;
}

extern "C" int ks_destroy(ks_loop_t h) {
    if (!h) return KS_OK;
    cudaSetDevice(h->dev);
    cudaDeviceSynchronize();
    for (auto& r : h->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->pool) cudaEventDestroy(e);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->side) cudaStreamDestroy(h->side);
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    if (h->gcap) cudaStreamDestroy(h->gcap);
    if (h->gcap2) cudaStreamDestroy(h->gcap2);
    if (h->gfork) cudaEventDestroy(h->gfork);
    if (h->gjoin) cudaEventDestroy(h->gjoin);
    for (void* p : h->allocs) cudaFree(p);
    delete h;
    return KS_OK;
}

extern "C" int ks_residual(ks_loop_t h, const void* u, const double* T, void* r, double* J,
                           void* stream) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!u || !T) return fail(KS_ERR_ARG, "u and T are required");
    cudaStream_t s = (cudaStream_t)stream;
    const int pr = h->api_prec;
    Work& w = h->api;
    KS_TRY(load_state(h, w, pr, u, T, s));
    if (pr == P64) KS_TRY(run_residual<double>(h, w, pr, s));
    else KS_TRY(run_residual<float>(h, w, pr, s));
    KS_TRY(run_finalize(h, w, w.T, pr, 0, s));
    const int B = h->d.B;
    if (r) {
        void* dst = is_device_ptr(r) ? r : w.io[pr];
        if (pr == P64) KS_TRY((run_synth<double, COL_SYNTH_R>(h, w, pr, (double*)dst, s)));
        else KS_TRY((run_synth<float, COL_SYNTH_R>(h, w, pr, (float*)dst, s)));
        if (dst != r) KS_TRY(copy_out(r, dst, (size_t)h->ngrid * elem_size(pr), s));
    }
    KS_TRY(copy_out(J, w.J, B * sizeof(double), s));
    if ((r && !is_device_ptr(r)) || (J && !is_device_ptr(J)) || !is_device_ptr(u))
        KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

extern "C" int ks_adjoint_grad(ks_loop_t h, const void* u, const double* T, void* G, double* dJdT,
                               void* stream) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!u || !T || !G) return fail(KS_ERR_ARG, "u, T and G are required");
    cudaStream_t s = (cudaStream_t)stream;
    const int pr = h->api_prec;
    Work& w = h->api;
    KS_TRY(load_state(h, w, pr, u, T, s));
    if (pr == P64) KS_TRY(run_gradient<double>(h, w, pr, s));
    else KS_TRY(run_gradient<float>(h, w, pr, s));
    KS_TRY(run_finalize(h, w, w.T, pr, 0, s));
    void* dst = is_device_ptr(G) ? G : w.io[pr];
    if (pr == P64) KS_TRY((run_synth<double, COL_SYNTH_G>(h, w, pr, (double*)dst, s)));
    else KS_TRY((run_synth<float, COL_SYNTH_G>(h, w, pr, (float*)dst, s)));
    if (dst != G) KS_TRY(copy_out(G, dst, (size_t)h->ngrid * elem_size(pr), s));
    KS_TRY(copy_out(dJdT, w.dJdT, h->d.B * sizeof(double), s));
    if (!is_device_ptr(G) || (dJdT && !is_device_ptr(dJdT)) || !is_device_ptr(u))
        KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

namespace {

// initial precision of the resident state
int start_prec(ks_loop* h) { return h->mode == KS_FP32 || h->mode == KS_MIXED ? P32 : P64; }

}  // namespace


// dst[b] = band of loop b in double, taken from the float band for loops running in float
__global__ void k_band_merge(const cpx<float>* s32, const cpx<double>* s64, cpx<double>* dst,
                             const long long* boff, const int* prec, int B, int nkx,
                             const int* ks) {
    const int b = blockIdx.y;
    if (b >= B) return;
    const long long n = (long long)nkx * (2 * ks[b] + 1);
    const long long o = boff[b];
    const bool f = prec[b] == 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        dst[o + i] = f ? mk<double>((double)s32[o + i].x, (double)s32[o + i].y) : s64[o + i];
    }
}

// dst[b] = src[b] (double bands) for the loops with sel[b]
__global__ void k_band_copy_sel(const cpx<double>* src, cpx<double>* dst, const long long* boff,
                                const int* sel, int B, int nkx, const int* ks) {
    const int b = blockIdx.y;
    if (b >= B || !sel[b]) return;
    const long long n = (long long)nkx * (2 * ks[b] + 1);
    const long long o = boff[b];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[o + i] = src[o + i];
}

// out[b] = cur[b] + (cur[b] - anc[b]) c_b for every loop (c_b = 0: out[b] = cur[b])
__global__ void k_band_extrap(const cpx<double>* cur, const cpx<double>* anc, const double* coef,
                              cpx<double>* out, const long long* boff, int B, int nkx,
                              const int* ks) {
    const int b = blockIdx.y;
    if (b >= B) return;
    const long long n = (long long)nkx * (2 * ks[b] + 1);
    const long long o = boff[b];
    const double c = coef[b];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cpx<double> v = cur[o + i];
        out[o + i] = (c == 0.0) ? v : v + scale(v - anc[o + i], c);
    }
}

// the double band src becomes the resident band of each selected loop, in the loop's precision
__global__ void k_band_store_sel(const cpx<double>* src, cpx<double>* s64, cpx<float>* s32,
                                 const long long* boff, const int* prec, const int* sel, int B,
                                 int nkx, const int* ks) {
    const int b = blockIdx.y;
    if (b >= B || !sel[b]) return;
    const long long n = (long long)nkx * (2 * ks[b] + 1);
    const long long o = boff[b];
    const bool f = prec[b] == 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cpx<double> v = src[o + i];
        if (f) s32[o + i] = mk<float>((float)v.x, (float)v.y);
        else s64[o + i] = v;
    }
}

namespace {

int set_state_full(ks_loop* h, const void* u, const double* T, cudaStream_t s) {
    const int B = h->d.B;
    Work& w = h->st;
    const int pr0 = start_prec(h);
    if (h->mode == KS_MIXED) {
        // the caller's field is double: project in double, round the band to float
        KS_TRY(load_state(h, w, P64, u, T, s));
        const long long n = h->nband;
        k_band_d2f<<<(int)std::min<long long>((n + 255) / 256, 152 * 8), 256, 0, s>>>(
            (const cpx<double>*)w.uh[P64], (cpx<float>*)w.uh[P32], n);
        KS_CUDA(cudaGetLastError());
    } else {
        KS_TRY(load_state(h, w, pr0, u, T, s));
    }
    KS_CUDA(cudaMemsetAsync(w.status, 0, B * sizeof(int), s));
    KS_CUDA(cudaMemsetAsync(w.steps, 0, B * sizeof(long long), s));
    KS_CUDA(cudaMemsetAsync(w.sqrtJ, 0, B * sizeof(double), s));
    h->h_prec.assign(B, pr0);
    KS_CUDA(cudaMemcpyAsync(w.prec, h->h_prec.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    h->h_status.assign(B, KS_RUNNING);
    h->h_steps.assign(B, 0);
    w.mix_valid[P64] = w.mix_valid[P32] = false;
    h->state_set = true;
    h->hist_steps.assign(B, {});
    h->hist_sqrtJ.assign(B, {});
    h->hist_prec.assign(B, {});
    h->anc_sq.assign(B, -1.0);
    h->anc_T.assign(B, 0.0);
    h->n_extrap = h->n_extrap_rejected = 0;
    return KS_OK;
}

// ---- graphs of the four-launch form ----
// The four launches of a tau-step depend on one another and on nothing the host computes between
// steps, so a run of `steps` (even) steps is captured once and replayed; an even run leaves the
// step parity where it found it.  While both precisions have live loops, the float and double
// chains of each step are independent (they touch disjoint loops) and the graph holds them as
// two parallel branches.
constexpr int kGraphSteps = 16;
constexpr size_t kGraphCache = 8;

int step_graph(ks_loop* h, Work& w, const bool* live, double tol, double swt, int steps,
               const ks_loop::StepGraph** out) {
    for (const auto& g : h->graphs)
        if (g.work == &w && g.live[0] == live[0] && g.live[1] == live[1] && g.tol == tol &&
            g.swt == swt && g.par == w.par && g.xi == h->xi && g.steps == steps) {
            *out = &g;
            return KS_OK;
        }
    if (!h->gcap) {
        KS_CUDA(cudaStreamCreateWithFlags(&h->gcap, cudaStreamNonBlocking));
        KS_CUDA(cudaStreamCreateWithFlags(&h->gcap2, cudaStreamNonBlocking));
        KS_CUDA(cudaEventCreateWithFlags(&h->gfork, cudaEventDisableTiming));
        KS_CUDA(cudaEventCreateWithFlags(&h->gjoin, cudaEventDisableTiming));
    }
    const bool both = live[P32] && live[P64];
    const int par0 = w.par;
    const long long l0 = h->launches;
    KS_CUDA(cudaStreamBeginCapture(h->gcap, cudaStreamCaptureModeThreadLocal));
    int rc = KS_OK;
    for (int i = 0; i < steps && rc == KS_OK; ++i) {
        cudaStream_t s64 = h->gcap;
        if (both) {
            if (cudaEventRecord(h->gfork, h->gcap) != cudaSuccess ||
                cudaStreamWaitEvent(h->gcap2, h->gfork, 0) != cudaSuccess) {
                rc = fail(KS_ERR_CUDA, "graph capture: fork failed");
                break;
            }
            s64 = h->gcap2;
        }
        if (live[P32]) rc = run_step<float>(h, w, P32, tol, swt, h->gcap);
        if (rc == KS_OK && live[P64]) rc = run_step<double>(h, w, P64, tol, 0.0, s64);
        if (rc == KS_OK && both &&
            (cudaEventRecord(h->gjoin, h->gcap2) != cudaSuccess ||
             cudaStreamWaitEvent(h->gcap, h->gjoin, 0) != cudaSuccess))
            rc = fail(KS_ERR_CUDA, "graph capture: join failed");
        w.par ^= 1;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->gcap, &graph);
    w.par = par0;
    ks_loop::StepGraph g{};
    g.launches = h->launches - l0;
    h->launches = l0;
    if (rc != KS_OK || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != KS_OK ? rc : fail(KS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    }
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    KS_CUDA(ei);
    g.work = &w;
    g.live[0] = live[0];
    g.live[1] = live[1];
    g.tol = tol;
    g.swt = swt;
    g.par = par0;
    g.xi = h->xi;
    g.steps = steps;
    if (h->graphs.size() >= kGraphCache) {
        KS_CUDA(cudaDeviceSynchronize());  // the oldest graph may still be replaying
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(g);
    *out = &h->graphs.back();
    return KS_OK;
}

// n tau-steps in the four-launch form of the precisions marked live (M primed): runs of even
// length as graph replays unless the knob is off or profiling is on, the rest launch by launch
int phase_steps(ks_loop* h, Work& w, const bool* live, long long n, double tol, double swt,
                cudaStream_t s) {
    long long i = 0;
    if (h->graph && !h->prof) {
        while (n - i >= 2) {
            const int G = (int)std::min<long long>(kGraphSteps, (n - i) & ~1LL);
            const ks_loop::StepGraph* g = nullptr;
            KS_TRY(step_graph(h, w, live, tol, swt, G, &g));
            for (const long long end = i + (n - i) / G * G; i < end; i += G) {
                KS_CUDA(cudaGraphLaunch(g->exec, s));
                h->launches += g->launches;
                h->graph_replays++;
            }
        }
    }
    for (; i < n; ++i) {
        if (live[P32]) KS_TRY(run_step<float>(h, w, P32, tol, swt, s));
        if (live[P64]) KS_TRY(run_step<double>(h, w, P64, tol, 0.0, s));
        w.par ^= 1;
    }
    return KS_OK;
}

constexpr long long kMaxPerLaunch = 1 << 14;

// n tau-steps of the live loops of precision pr in launch form `form` (form_of), starting from
// w.par and leaving it advanced by n.  adj32: a double cluster form of a KS_MIXED handle may
// form the adjoint in float (the "finish_f32_adjoint" knob).
int form_steps(ks_loop* h, Work& w, int pr, int form, long long n, double tol, double swt,
               cudaStream_t s, bool adj32) {
    if (form == 2) {
        const bool live[2] = {pr == P64, pr == P32};
        if (!w.mix_valid[pr]) {
            if (pr == P64) KS_TRY(run_prime<double>(h, w, pr, s));
            else KS_TRY(run_prime<float>(h, w, pr, s));
        }
        return phase_steps(h, w, live, n, tol, pr == P32 ? swt : 0.0, s);
    }
    for (long long done = 0; done < n;) {
        const long long c = std::min(kMaxPerLaunch, n - done);
        if (form == 0) {
            if (pr == P32)
                KS_TRY((run_cluster<float, float>(h, w, P32, c, tol, swt, s)));
            else if (adj32 && h->mode == KS_MIXED && h->finish_f32_adjoint && h->cplan[2].bytes > 0)
                KS_TRY((run_cluster<double, float>(h, w, P64, c, tol, 0.0, s)));
            else
                KS_TRY((run_cluster<double, double>(h, w, P64, c, tol, 0.0, s)));
        } else {
            if (!w.mix_valid[pr]) {
                if (pr == P64) KS_TRY(run_prime<double>(h, w, pr, s));
                else KS_TRY(run_prime<float>(h, w, pr, s));
            }
            if (pr == P32) KS_TRY(run_persist<float>(h, w, P32, c, tol, swt, s));
            else KS_TRY(run_persist<double>(h, w, P64, c, tol, 0.0, s));
        }
        if (c & 1) w.par ^= 1;
        done += c;
    }
    return KS_OK;
}

// destroy the cached graphs once no replay of them can still be queued on any stream
void drop_graphs(ks_loop* h) {
    if (h->graphs.empty()) return;
    cudaDeviceSynchronize();
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

// run n steps of the resident state on the precisions that have live loops.  The loops of the
// two precisions are disjoint and independent, so each precision may take its own launch form
// and run its n steps from the same parity; where both take the cluster form (and profiling is
// off) the double launch runs beside the float one on the side stream, where both take the
// four-launch form their graphs hold the two chains as parallel branches.
int steps_impl(ks_loop* h, long long n, double tol, cudaStream_t s, bool device_switch = true) {
    Work& w = h->st;
    bool live[2] = {false, false};
    for (int b = 0; b < h->d.B; ++b)
        if (h->h_status[b] == KS_RUNNING) live[h->h_prec[b]] = true;
    const double swt = (h->mode == KS_MIXED && device_switch) ? h->switch_tol : 0.0;
    const int form[2] = {form_of(h, P64), form_of(h, P32)};
    if (live[P32] && live[P64] && form[P32] == 2 && form[P64] == 2) {
        for (int pr = 0; pr < 2; ++pr)
            if (!w.mix_valid[pr]) {
                if (pr == P64) KS_TRY(run_prime<double>(h, w, pr, s));
                else KS_TRY(run_prime<float>(h, w, pr, s));
            }
        return phase_steps(h, w, live, n, tol, swt, s);
    }
    if (live[P32] && live[P64] && form[P32] == 0 && form[P64] == 0 && !h->prof) {
        // each launch carries T forward only for the frozen loops of its own precision (a loop
        // that freezes during the chunk is written by its own kernel alone)
        if (!h->side) {
            KS_CUDA(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
            KS_CUDA(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
            KS_CUDA(cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming));
        }
        for (long long done = 0; done < n;) {
            const long long c = std::min(kMaxPerLaunch, n - done);
            KS_CUDA(cudaEventRecord(h->fork, s));
            KS_CUDA(cudaStreamWaitEvent(h->side, h->fork, 0));
            KS_TRY((run_cluster<float, float>(h, w, P32, c, tol, swt, s, true)));
            if (h->mode == KS_MIXED && h->finish_f32_adjoint && h->cplan[2].bytes > 0)
                KS_TRY((run_cluster<double, float>(h, w, P64, c, tol, 0.0, h->side, true)));
            else
                KS_TRY((run_cluster<double, double>(h, w, P64, c, tol, 0.0, h->side, true)));
            KS_CUDA(cudaEventRecord(h->join, h->side));
            KS_CUDA(cudaStreamWaitEvent(s, h->join, 0));
            if (c & 1) w.par ^= 1;
            done += c;
        }
        return KS_OK;
    }
    // one precision at a time, each from the same parity
    const int par0 = w.par;
    for (int pr : {P32, P64}) {
        if (!live[pr]) continue;
        w.par = par0;
        KS_TRY(form_steps(h, w, pr, form[pr], n, tol, swt, s, true));
    }
    w.par = par0 ^ (int)(n & 1);
    return KS_OK;
}

int readback(ks_loop* h, cudaStream_t s) {
    Work& w = h->st;
    const int B = h->d.B;
    KS_CUDA(cudaMemcpyAsync(h->h_status.data(), w.status, B * sizeof(int), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaMemcpyAsync(h->h_sqrtJ.data(), w.sqrtJ, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaMemcpyAsync(h->h_steps.data(), w.steps, B * sizeof(long long), cudaMemcpyDeviceToHost, s));
    int err = 0;
    KS_CUDA(cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    if (err) {
        // a bounded wait gave up (a grid barrier of the persistent kernel, or an exchange of the
        // cluster kernel): clear the barrier for the next launch and report it
        KS_CUDA(cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned int), s));
        KS_CUDA(cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
        KS_CUDA(cudaStreamSynchronize(s));
        return fail(KS_ERR_TIMEOUT, "a bounded wait timed out (grid barrier or cluster exchange)");
    }
    return KS_OK;
}

// move the loops flagged in sel (host) from float to double
int switch_to_double(ks_loop* h, const std::vector<int>& sel, cudaStream_t s) {
    Work& w = h->st;
    const int B = h->d.B;
    KS_CUDA(cudaMemcpyAsync(w.sel, sel.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    dim3 g(8, B);
    k_band_f2d<<<g, 256, 0, s>>>((const cpx<float>*)w.uh[P32], (cpx<double>*)w.uh[P64], h->d_boff,
                                 w.sel, B, h->d.nkx, h->d_ks);
    KS_CUDA(cudaGetLastError());
    for (int b = 0; b < B; ++b)
        if (sel[b]) {
            h->h_prec[b] = P64;
            h->h_status[b] = KS_RUNNING;
        }
    KS_CUDA(cudaMemcpyAsync(w.prec, h->h_prec.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    KS_CUDA(cudaMemcpyAsync(w.status, h->h_status.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    w.mix_valid[P64] = false;
    return KS_OK;
}

int set_status(ks_loop* h, cudaStream_t s) {
    KS_CUDA(cudaMemcpyAsync(h->st.status, h->h_status.data(), h->d.B * sizeof(int),
                            cudaMemcpyHostToDevice, s));
    return KS_OK;
}

// evaluate J at the current resident state of every loop (per precision) into sqrtJ
int final_eval(ks_loop* h, cudaStream_t s) {
    Work& w = h->st;
    for (int pr = 0; pr < 2; ++pr) {
        if (!h->need[pr]) continue;
        bool any = false;
        for (int b = 0; b < h->d.B; ++b) any |= (h->h_prec[b] == pr);
        if (!any) continue;
        const double* Tc = w.T + (size_t)w.par * h->d.B;
        if (pr == P64) KS_TRY(run_residual<double>(h, w, pr, s));
        else KS_TRY(run_residual<float>(h, w, pr, s));
        KS_TRY(run_finalize(h, w, Tc, pr, 1, s));
    }
    return KS_OK;
}

// sqrt(J) of the resident state of every loop evaluated in double (the band of float loops
// widened first): the residual evaluation of a mixed descent stays in double.  Uses the API
// workspace; the resident state is not touched.
// double_band: evaluate the double band of every loop instead (the projected input right after
// ks_set_state of a mixed handle, before any float step)
int monitor_f64(ks_loop* h, cudaStream_t s, std::vector<double>& out, bool double_band = false) {
    Work& w = h->st;
    Work& a = h->api;
    const int B = h->d.B;
    dim3 g(8, B);
    const int* sel_prec = w.prec;
    if (double_band) {
        KS_CUDA(cudaMemsetAsync(w.sel, 0, B * sizeof(int), s));  // precision 0 (double) for all
        sel_prec = w.sel;
    }
    k_band_merge<<<g, 256, 0, s>>>((const cpx<float>*)w.uh[P32], (const cpx<double>*)w.uh[P64],
                                   (cpx<double>*)a.uh[P64], h->d_boff, sel_prec, B, h->d.nkx, h->d_ks);
    KS_CUDA(cudaGetLastError());
    KS_CUDA(cudaMemcpyAsync(a.T, w.T + (size_t)w.par * B, B * sizeof(double), cudaMemcpyDeviceToDevice, s));
    a.par = 0;
    k_prep_wT<<<(B + 127) / 128, 128, 0, s>>>(a.T, a.wT, B);
    KS_CUDA(cudaGetLastError());
    KS_TRY(run_residual<double>(h, a, P64, s));
    KS_TRY(run_finalize(h, a, a.T, P64, 0, s));
    out.resize(B);
    KS_CUDA(cudaMemcpyAsync(out.data(), a.sqrtJ, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

// Probe of the float floor of a mixed descent.  The loops flagged in sel take n double steps from
// their current state (the float band widened exactly) on the API workspace; the resident state
// is not touched.  out[b] gets sqrt(J) of each probed loop after those steps, evaluated in
// double, and Tout[b] its period.  A float state carries rounding noise that the double steps
// remove within a few hundred steps; what remains is the part of the residual the float steps
// can still reduce, so comparing it with sqrt(J) of the float state tells a float phase that
// still converges (beneath its noise) from one that has stalled.
int polish_probe(ks_loop* h, cudaStream_t s, const std::vector<int>& sel, long long n,
                 std::vector<double>& out, std::vector<double>& Tout) {
    Work& w = h->st;
    Work& a = h->api;
    const int B = h->d.B;
    dim3 g(8, B);
    k_band_merge<<<g, 256, 0, s>>>((const cpx<float>*)w.uh[P32], (const cpx<double>*)w.uh[P64],
                                   (cpx<double>*)a.uh[P64], h->d_boff, w.prec, B, h->d.nkx, h->d_ks);
    KS_CUDA(cudaGetLastError());
    KS_CUDA(cudaMemcpyAsync(a.T, w.T + (size_t)w.par * B, B * sizeof(double), cudaMemcpyDeviceToDevice, s));
    a.par = 0;
    k_prep_wT<<<(B + 127) / 128, 128, 0, s>>>(a.T, a.wT, B);
    KS_CUDA(cudaGetLastError());
    std::vector<int> st(B), pr(B, P64);
    for (int b = 0; b < B; ++b) st[b] = sel[b] ? KS_RUNNING : KS_STEP_CAP;
    KS_CUDA(cudaMemcpyAsync(a.status, st.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    KS_CUDA(cudaMemcpyAsync(a.prec, pr.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    KS_CUDA(cudaMemsetAsync(a.steps, 0, B * sizeof(long long), s));
    a.mix_valid[P64] = false;
    KS_TRY(form_steps(h, a, P64, form_of(h, P64), n, 0.0, 0.0, s, false));
    const double* Tc = a.T + (size_t)a.par * B;
    KS_TRY(run_residual<double>(h, a, P64, s));
    KS_TRY(run_finalize(h, a, Tc, P64, 0, s));
    out.resize(B);
    Tout.resize(B);
    KS_CUDA(cudaMemcpyAsync(out.data(), a.sqrtJ, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaMemcpyAsync(Tout.data(), Tc, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

// The loops flagged in sel continue in double from the state the last polish_probe left in the
// API workspace (band, T after n more steps, step counters advanced by n).
int switch_polished(ks_loop* h, cudaStream_t s, const std::vector<int>& sel, long long n,
                    const std::vector<double>& Tp) {
    Work& w = h->st;
    Work& a = h->api;
    const int B = h->d.B;
    dim3 g(8, B);
    KS_CUDA(cudaMemcpyAsync(w.sel, sel.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    k_band_copy_sel<<<g, 256, 0, s>>>((const cpx<double>*)a.uh[P64], (cpx<double>*)w.uh[P64],
                                      h->d_boff, w.sel, B, h->d.nkx, h->d_ks);
    KS_CUDA(cudaGetLastError());
    std::vector<double> Tcur(B), wTcur(B);
    KS_CUDA(cudaMemcpyAsync(Tcur.data(), w.T + (size_t)w.par * B, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaMemcpyAsync(wTcur.data(), w.wT + (size_t)w.par * B, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < B; ++b)
        if (sel[b]) {
            Tcur[b] = Tp[b];
            wTcur[b] = 2.0 * 3.14159265358979323846 / Tp[b];
            h->h_prec[b] = P64;
            h->h_status[b] = KS_RUNNING;
            h->h_steps[b] += n;
            h->anc_sq[b] = -1.0;  // an extrapolation anchor from the float phase no longer applies
        }
    KS_CUDA(cudaMemcpyAsync(w.T + (size_t)w.par * B, Tcur.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
    KS_CUDA(cudaMemcpyAsync(w.wT + (size_t)w.par * B, wTcur.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
    KS_CUDA(cudaMemcpyAsync(w.prec, h->h_prec.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    KS_CUDA(cudaMemcpyAsync(w.status, h->h_status.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    KS_CUDA(cudaMemcpyAsync(w.steps, h->h_steps.data(), B * sizeof(long long), cudaMemcpyHostToDevice, s));
    w.mix_valid[P64] = false;
    return KS_OK;
}

// One extrapolation round of App. C over the running loops, from sqrt(J) of the current states
// (val, evaluated in double).  A loop below extrap_start without an anchor takes its current
// state as the anchor; a loop whose sqrt(J) has fallen to half its anchor's is extrapolated
// geometrically, l* ~ l + (l - l_a) rho / (1 - rho), rho = sqrt(J) / sqrt(J_a), on the band and
// T.  The candidate is kept only if its sqrt(J), evaluated in double, is lower; either way the
// loop's anchor moves to the state it continues from.  touched[b] marks the loops handled.
// The start threshold and the drop ratio are the handle's knobs; their defaults, 1e-3 and
// 1/2, are the values of the example of App. C.

int extrapolate_round(ks_loop* h, cudaStream_t s, const std::vector<double>& val,
                      std::vector<char>& touched) {
    Work& w = h->st;
    Work& a = h->api;
    const int B = h->d.B;
    const long long nb = h->nband;
    if (!h->anc) {
        void* p = nullptr;
        KS_TRY(dev_alloc(h, &p, nb * sizeof(cpx<double>)));
        h->anc = (double*)p;
        KS_TRY(dev_alloc(h, &p, nb * sizeof(cpx<double>)));
        h->cand = (double*)p;
        KS_TRY(dev_alloc(h, &p, B * sizeof(double)));
        h->coef = (double*)p;
        KS_TRY(dev_alloc(h, &p, 3 * B * sizeof(int)));
        h->esel = (int*)p;
    }
    std::vector<double> Tcur(B), wTcur(B);
    KS_CUDA(cudaMemcpyAsync(Tcur.data(), w.T + (size_t)w.par * B, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaMemcpyAsync(wTcur.data(), w.wT + (size_t)w.par * B, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    dim3 g(8, B);
    k_band_merge<<<g, 256, 0, s>>>((const cpx<float>*)w.uh[P32], (const cpx<double>*)w.uh[P64],
                                   (cpx<double>*)h->cand, h->d_boff, w.prec, B, h->d.nkx, h->d_ks);
    KS_CUDA(cudaGetLastError());
    KS_CUDA(cudaStreamSynchronize(s));
    std::vector<int> selA(B, 0), selAcc(B, 0), selRej(B, 0);
    std::vector<double> c(B, 0.0), Tc(Tcur);
    bool anyA = false, anyC = false;
    for (int b = 0; b < B; ++b) {
        if (h->h_status[b] != KS_RUNNING || !(val[b] <= h->extrap_start)) continue;
        if (h->anc_sq[b] < 0.0) {
            selA[b] = 1;
            h->anc_sq[b] = val[b];
            h->anc_T[b] = Tcur[b];
            anyA = true;
            continue;
        }
        if (val[b] > h->extrap_drop * h->anc_sq[b]) continue;
        const double rho = val[b] / h->anc_sq[b];
        c[b] = rho / (1.0 - rho);
        Tc[b] = Tcur[b] + (Tcur[b] - h->anc_T[b]) * c[b];
        anyC = true;
    }
    if (anyA) {
        KS_CUDA(cudaMemcpyAsync(h->esel, selA.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
        k_band_copy_sel<<<g, 256, 0, s>>>((const cpx<double>*)h->cand, (cpx<double>*)h->anc,
                                          h->d_boff, h->esel, B, h->d.nkx, h->d_ks);
        KS_CUDA(cudaGetLastError());
    }
    if (!anyC) {
        KS_CUDA(cudaStreamSynchronize(s));
        return KS_OK;
    }
    // candidates into the API workspace, their sqrt(J) in double
    KS_CUDA(cudaMemcpyAsync(h->coef, c.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
    k_band_extrap<<<g, 256, 0, s>>>((const cpx<double>*)h->cand, (const cpx<double>*)h->anc,
                                    h->coef, (cpx<double>*)a.uh[P64], h->d_boff, B, h->d.nkx,
                                    h->d_ks);
    KS_CUDA(cudaGetLastError());
    KS_CUDA(cudaMemcpyAsync(a.T, Tc.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
    a.par = 0;
    k_prep_wT<<<(B + 127) / 128, 128, 0, s>>>(a.T, a.wT, B);
    KS_CUDA(cudaGetLastError());
    KS_TRY(run_residual<double>(h, a, P64, s));
    KS_TRY(run_finalize(h, a, a.T, P64, 0, s));
    std::vector<double> sqe(B);
    KS_CUDA(cudaMemcpyAsync(sqe.data(), a.sqrtJ, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    KS_CUDA(cudaStreamSynchronize(s));
    bool anyAcc = false, anyRej = false;
    for (int b = 0; b < B; ++b) {
        if (c[b] == 0.0) continue;
        touched[b] = 1;
        if (sqe[b] == sqe[b] && sqe[b] < val[b]) {
            selAcc[b] = 1;
            anyAcc = true;
            h->anc_sq[b] = sqe[b];
            h->anc_T[b] = Tc[b];
            Tcur[b] = Tc[b];
            wTcur[b] = 2.0 * 3.14159265358979323846 / Tc[b];
            ++h->n_extrap;
        } else {
            selRej[b] = 1;
            anyRej = true;
            h->anc_sq[b] = val[b];
            h->anc_T[b] = Tcur[b];
            ++h->n_extrap_rejected;
        }
    }
    if (anyAcc) {
        KS_CUDA(cudaMemcpyAsync(h->esel + B, selAcc.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
        k_band_store_sel<<<g, 256, 0, s>>>((const cpx<double>*)a.uh[P64], (cpx<double>*)w.uh[P64],
                                           (cpx<float>*)w.uh[P32], h->d_boff, w.prec, h->esel + B,
                                           B, h->d.nkx, h->d_ks);
        KS_CUDA(cudaGetLastError());
        k_band_copy_sel<<<g, 256, 0, s>>>((const cpx<double>*)a.uh[P64], (cpx<double>*)h->anc,
                                          h->d_boff, h->esel + B, B, h->d.nkx, h->d_ks);
        KS_CUDA(cudaGetLastError());
        KS_CUDA(cudaMemcpyAsync(w.T + (size_t)w.par * B, Tcur.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
        KS_CUDA(cudaMemcpyAsync(w.wT + (size_t)w.par * B, wTcur.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
        w.mix_valid[P64] = w.mix_valid[P32] = false;  // the mixed values derive from the band
    }
    if (anyRej) {
        KS_CUDA(cudaMemcpyAsync(h->esel + 2 * B, selRej.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
        k_band_copy_sel<<<g, 256, 0, s>>>((const cpx<double>*)h->cand, (cpx<double>*)h->anc,
                                          h->d_boff, h->esel + 2 * B, B, h->d.nkx, h->d_ks);
        KS_CUDA(cudaGetLastError());
    }
    KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

// write the resident state to u (grid) in the handle's I/O precision
int get_state_impl(ks_loop* h, void* u, double* T, cudaStream_t s) {
    Work& w = h->st;
    const int B = h->d.B;
    if (u) {
        if (h->mode == KS_MIXED) {
            // gather both precisions into the double band of the API workspace, synthesise there
            Work& a = h->api;
            dim3 g(8, B);
            k_band_merge<<<g, 256, 0, s>>>((const cpx<float>*)w.uh[P32], (const cpx<double>*)w.uh[P64],
                                           (cpx<double>*)a.uh[P64], h->d_boff, w.prec, B, h->d.nkx,
                                           h->d_ks);
            KS_CUDA(cudaGetLastError());
            void* dst = is_device_ptr(u) ? u : a.io[P64];
            KS_TRY((run_synth<double, COL_SYNTH_U>(h, a, P64, (double*)dst, s)));
            if (dst != u) KS_TRY(copy_out(u, dst, (size_t)h->ngrid * sizeof(double), s));
        } else {
            const int pr = (h->mode == KS_FP32) ? P32 : P64;
            void* dst = is_device_ptr(u) ? u : w.io[pr];
            if (pr == P64) KS_TRY((run_synth<double, COL_SYNTH_U>(h, w, pr, (double*)dst, s)));
            else KS_TRY((run_synth<float, COL_SYNTH_U>(h, w, pr, (float*)dst, s)));
            if (dst != u) KS_TRY(copy_out(u, dst, (size_t)h->ngrid * elem_size(pr), s));
        }
    }
    if (T) KS_TRY(copy_out(T, w.T + (size_t)w.par * B, B * sizeof(double), s));
    return KS_OK;
}

}  // namespace

extern "C" int ks_set_state(ks_loop_t h, const void* u, const double* T, void* stream) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!u || !T) return fail(KS_ERR_ARG, "u and T are required");
    cudaStream_t s = (cudaStream_t)stream;
    KS_TRY(set_state_full(h, u, T, s));
    if (!is_device_ptr(u) || !is_device_ptr(T)) KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

extern "C" int ks_step(ks_loop_t h, long long nsteps, double tol, void* stream) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!h->state_set) return fail(KS_ERR_STATE, "ks_step before ks_set_state");
    if (nsteps < 0) return fail(KS_ERR_ARG, "nsteps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const double t = tol < 0.0 ? h->tol : tol;
    KS_TRY(steps_impl(h, nsteps, t, s));
    if (h->mode == KS_MIXED) {
        // hand loops that met the switch criterion to the double kernels
        KS_TRY(readback(h, s));
        std::vector<int> sel(h->d.B, 0);
        bool any = false;
        for (int b = 0; b < h->d.B; ++b)
            if (h->h_status[b] == ST_SWITCH) {
                sel[b] = 1;
                any = true;
            }
        if (any) KS_TRY(switch_to_double(h, sel, s));
    }
    return KS_OK;
}

extern "C" int ks_get_state(ks_loop_t h, void* u, double* T, long long* steps, double* sqrtJ,
                            int* status, void* stream) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!h->state_set) return fail(KS_ERR_STATE, "ks_get_state before ks_set_state");
    cudaStream_t s = (cudaStream_t)stream;
    KS_TRY(readback(h, s));
    KS_TRY(get_state_impl(h, u, T, s));
    const int B = h->d.B;
    Work& w = h->st;
    KS_TRY(copy_out(steps, w.steps, B * sizeof(long long), s));
    KS_TRY(copy_out(sqrtJ, w.sqrtJ, B * sizeof(double), s));
    if (status) {
        // report the internal switch marker as running
        std::vector<int> st = h->h_status;
        for (int& v : st)
            if (v == ST_SWITCH) v = KS_RUNNING;
        KS_CUDA(cudaMemcpyAsync(status, st.data(), B * sizeof(int), cudaMemcpyDefault, s));
    }
    KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

extern "C" int ks_descend(ks_loop_t h, void* u, double* T, long long max_steps, double tol,
                          long long* steps, double* sqrtJ, int* status, void* stream) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!u || !T) return fail(KS_ERR_ARG, "u and T are required");
    cudaStream_t s = (cudaStream_t)stream;
    const long long cap = max_steps < 0 ? h->max_steps : max_steps;
    const double tl = tol < 0.0 ? h->tol : tol;
    const int B = h->d.B;
    KS_TRY(set_state_full(h, u, T, s));
    // stall detection: sqrt(J) at the start of the current window
    std::vector<double> win_val(B, -1.0);
    std::vector<long long> win_step(B, 0);
    std::vector<double> mon;
    // mixed descents: the float kernels do not switch on their own; the switch is decided here
    // from sqrt(J) evaluated in double, which keeps falling after the float value has reached
    // its noise floor
    const bool monitor = (h->mode == KS_MIXED);
    // float-floor probe (knob "switch_probe"): the rate of the float phase in decades of sqrt(J)
    // per step over windows of stall_window / 4 steps, the best rate over windows that lie in the
    // tail (sqrt(J) < 1e-2 at their start), and the probe schedule.  When the rate falls below an
    // eighth of the best, a probe polishes a copy of the loop in double (polish_probe) and the
    // loop stays in float or switches from the polished copy (see the decision below).
    std::vector<double> rv0(B, -1.0), rbest(B, 0.0), rlast(B, 0.0);
    std::vector<long long> rs0(B, 0), pnext(B, 0);
    if (monitor) {
        // a loop whose float rounding alone already doubles sqrt(J) (it starts below the float
        // floor, e.g. a nearly converged loop) descends in double from the start
        std::vector<double> jf, jd;
        KS_TRY(monitor_f64(h, s, jf));
        KS_TRY(monitor_f64(h, s, jd, true));
        bool any = false;
        for (int b = 0; b < B; ++b)
            if (jf[b] > 2.0 * jd[b]) {
                h->h_prec[b] = P64;
                any = true;
            }
        if (any) {
            KS_CUDA(cudaMemcpyAsync(h->st.prec, h->h_prec.data(), B * sizeof(int),
                                    cudaMemcpyHostToDevice, s));
            h->st.mix_valid[P64] = false;
        }
    }
    long long done = 0;
    while (done < cap) {
        const long long c = std::min<long long>(h->chunk, cap - done);
        KS_TRY(steps_impl(h, c, tl, s, !monitor));
        done += c;
        KS_TRY(readback(h, s));
        if (monitor || h->extrapolate) KS_TRY(monitor_f64(h, s, mon));
        std::vector<double> val(B);
        for (int b = 0; b < B; ++b)
            val[b] = ((monitor && h->h_prec[b] == P32) || h->extrapolate) ? mon[b] : h->h_sqrtJ[b];
        for (int b = 0; b < B; ++b) {
            if (!h->hist_steps[b].empty() && h->hist_steps[b].back() == h->h_steps[b]) continue;
            h->hist_steps[b].push_back(h->h_steps[b]);
            h->hist_sqrtJ[b].push_back(val[b]);
            h->hist_prec[b].push_back(h->h_prec[b]);
        }
        std::vector<int> sel(B, 0), psel(B, 0);
        bool any_switch = false, any_live = false, status_dirty = false, any_probe = false;
        for (int b = 0; b < B; ++b) {
            int& stb = h->h_status[b];
            if (stb == ST_SWITCH) {
                sel[b] = 1;
                any_switch = true;
                continue;
            }
            if (stb != KS_RUNNING) continue;
            const double v = val[b];
            if (monitor && h->h_prec[b] == P32) {
                if (!(v == v) || v > 1e150) {
                    stb = KS_DIVERGED;
                    status_dirty = true;
                    continue;
                }
                if (v < tl) {
                    stb = KS_CONVERGED;  // the float loop already meets tol in double
                    status_dirty = true;
                    continue;
                }
                if (h->switch_tol > 0.0 && v <= h->switch_tol) {
                    sel[b] = 1;
                    any_switch = true;
                    continue;
                }
                if (h->switch_probe) {
                    const long long wr = std::max<long long>(1, h->stall_window / 4);
                    if (rv0[b] < 0.0) {
                        rv0[b] = v;
                        rs0[b] = h->h_steps[b];
                    } else if (h->h_steps[b] - rs0[b] >= wr) {
                        const double rate = std::log10(rv0[b] / v) / (double)(h->h_steps[b] - rs0[b]);
                        const bool tail = rv0[b] < 1e-2;  // the whole window in the tail
                        const bool bent = tail && rbest[b] > 0.0 && rate < 0.125 * rbest[b];
                        if (tail && rate > rbest[b]) rbest[b] = rate;
                        rlast[b] = rate;
                        rv0[b] = v;
                        rs0[b] = h->h_steps[b];
                        if (bent && h->h_steps[b] >= pnext[b]) {
                            psel[b] = 1;
                            any_probe = true;
                        }
                    }
                }
            }
            // no-progress test over a window of stall_window steps
            if (win_val[b] < 0.0) {
                win_val[b] = v;
                win_step[b] = h->h_steps[b];
            } else if (h->h_steps[b] - win_step[b] >= h->stall_window) {
                if (v > (1.0 - h->stall_drop) * win_val[b]) {
                    if (h->mode == KS_MIXED && h->h_prec[b] == P32) {
                        sel[b] = 1;
                        any_switch = true;
                    } else {
                        stb = KS_STALLED;
                        status_dirty = true;
                    }
                }
                win_val[b] = v;
                win_step[b] = h->h_steps[b];
            }
            if (stb == KS_RUNNING && !sel[b]) any_live = true;
        }
        if (any_probe) {
            std::vector<double> pv, pT;
            KS_TRY(polish_probe(h, s, psel, h->probe_steps, pv, pT));
            std::vector<int> ssel(B, 0);
            bool any_polished = false;
            for (int b = 0; b < B; ++b) {
                if (!psel[b]) continue;
                // The polish removes the float rounding noise.  Against what its steps would
                // give at the best tail rate: if it removes a fifth or more of sqrt(J), the float
                // state's value is mostly that noise and the float steps keep converging beneath
                // it (the stall window ends the float phase, no further probe); if it removes
                // less and descends at least four times faster than the float phase does now,
                // the float arithmetic holds the descent back: switch from the polished copy;
                // otherwise the bend was the loop's own dynamics (probe again at a later bend).
                const double expect = val[b] * std::pow(10.0, -rbest[b] * (double)h->probe_steps);
                const double removed = 1.0 - pv[b] / expect;
                const double rp = std::log10(val[b] / pv[b]) / (double)h->probe_steps;
                const bool go = removed < 0.2 && rp > 4.0 * std::max(rlast[b], 0.0);
                const long long wait = removed >= 0.2 ? (1LL << 62) : h->stall_window;
                if (go && pv[b] == pv[b] && pT[b] > 0.0) {
                    ssel[b] = 1;
                    sel[b] = 0;
                    any_polished = true;
                } else {
                    pnext[b] = h->h_steps[b] + wait;
                }
            }
            if (any_polished) {
                KS_TRY(switch_polished(h, s, ssel, h->probe_steps, pT));
                for (int b = 0; b < B; ++b)
                    if (ssel[b]) {
                        win_val[b] = -1.0;
                        any_live = true;
                    }
            }
        }
        if (any_switch) {
            KS_TRY(switch_to_double(h, sel, s));
            for (int b = 0; b < B; ++b)
                if (sel[b]) {
                    win_val[b] = -1.0;
                    any_live = true;
                }
        }
        if (status_dirty) KS_TRY(set_status(h, s));
        if (h->extrapolate && any_live) {
            std::vector<char> touched(B, 0);
            KS_TRY(extrapolate_round(h, s, val, touched));
            for (int b = 0; b < B; ++b)
                if (touched[b]) win_val[b] = -1.0;  // sqrt(J) moved by a jump: restart the window
        }
        if (!any_live) break;
    }
    // final residual at the resident state (in double for every loop of a mixed descent),
    // step-cap status for the loops still running
    KS_TRY(final_eval(h, s));
    KS_TRY(readback(h, s));
    if (monitor) {
        KS_TRY(monitor_f64(h, s, mon));
        KS_CUDA(cudaMemcpyAsync(h->st.sqrtJ, mon.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    for (int b = 0; b < B; ++b)
        if (h->h_status[b] == KS_RUNNING || h->h_status[b] == ST_SWITCH) h->h_status[b] = KS_STEP_CAP;
    KS_TRY(set_status(h, s));
    KS_TRY(get_state_impl(h, u, T, s));
    Work& w = h->st;
    KS_TRY(copy_out(steps, w.steps, B * sizeof(long long), s));
    KS_TRY(copy_out(sqrtJ, w.sqrtJ, B * sizeof(double), s));
    KS_TRY(copy_out(status, w.status, B * sizeof(int), s));
    KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

extern "C" int ks_profile(ks_loop_t h, int enable) {
    g_err.clear();
    KS_TRY(check_handle(h));
    h->prof = enable != 0;
    return KS_OK;
}

extern "C" int ks_profile_read(ks_loop_t h, int n, char* names, double* ms, long long* launches,
                               long long* total_launches, int reset) {
    g_err.clear();
    KS_TRY(check_handle(h));
    for (auto& r : h->pending) {
        KS_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        KS_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        h->kind_ms[r.kind] += (double)t;
        h->kind_count[r.kind] += 1;
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->pending.clear();
    const int k = (int)h->kind_names.size();
    for (int i = 0; i < k && i < n; ++i) {
        if (names) {
            std::strncpy(names + (size_t)i * 48, h->kind_names[i].c_str(), 47);
            names[(size_t)i * 48 + 47] = 0;
        }
        if (ms) ms[i] = h->kind_ms[i];
        if (launches) launches[i] = h->kind_count[i];
    }
    if (total_launches) *total_launches = h->launches;
    if (reset) {
        for (auto& v : h->kind_ms) v = 0.0;
        for (auto& v : h->kind_count) v = 0;
        h->launches = 0;
    }
    return k;
}

extern "C" int ks_set_option(ks_loop_t h, const char* key, long long value) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!key) return fail(KS_ERR_ARG, "null option name");
    const std::string k(key);
    if (k == "persistent") {
        h->path[P64] = h->path[P32] = value ? 1 : 2;
    } else if (k == "path" || k == "path_f64" || k == "path_f32") {
        if (value < 0 || value > 2) return fail(KS_ERR_ARG, "path must be 0, 1 or 2");
        if (k != "path_f32") h->path[P64] = (int)value;
        if (k != "path_f64") h->path[P32] = (int)value;
    } else if (k == "cluster") {
        if (value < 0 || value > 16) return fail(KS_ERR_ARG, "cluster must be 0 (auto) or 1..16");
        h->force_cluster = (int)value;
        KS_TRY((setup_cluster<double, double>(h)));
        KS_TRY((setup_cluster<float, float>(h)));
        if (h->mode == KS_MIXED) KS_TRY((setup_cluster<double, float>(h)));
        if (value && (h->cplan[0].C != value && h->cplan[1].C != value))
            return fail(KS_ERR_ARG, "requested cluster size does not fit this batch");
    } else if (k == "cluster_min_blocks") {
        if (value < 0 || value > 2) return fail(KS_ERR_ARG, "cluster_min_blocks must be 0 (auto), 1 or 2");
        h->force_mb = (int)value;
        KS_TRY((setup_cluster<double, double>(h)));
        KS_TRY((setup_cluster<float, float>(h)));
        if (h->mode == KS_MIXED) KS_TRY((setup_cluster<double, float>(h)));
    } else if (k == "cluster_exchange") {
        h->cexchange = value ? 1 : 0;
        KS_TRY((setup_cluster<double, double>(h)));
        KS_TRY((setup_cluster<float, float>(h)));
        if (h->mode == KS_MIXED) KS_TRY((setup_cluster<double, float>(h)));
    } else if (k == "test_barrier_timeout") {
        h->test_barrier_extra = value ? 1 : 0;
    } else if (k == "finish_f32_adjoint") {
        h->finish_f32_adjoint = value != 0;
    } else if (k == "switch_probe") {
        h->switch_probe = value ? 1 : 0;
    } else if (k == "switch_probe_steps") {
        if (value < 1 || value > 1000000) return fail(KS_ERR_ARG, "switch_probe_steps in [1, 1e6]");
        h->probe_steps = value;
    } else if (k == "extrapolate") {
        h->extrapolate = value ? 1 : 0;
    } else if (k == "extrapolate_start_ppm") {
        if (value < 1 || value > 1000000000LL) return fail(KS_ERR_ARG, "extrapolate_start_ppm in [1, 1e9]");
        h->extrap_start = (double)value * 1e-6;
    } else if (k == "extrapolate_drop_ppm") {
        if (value < 1 || value >= 1000000) return fail(KS_ERR_ARG, "extrapolate_drop_ppm in [1, 1e6)");
        h->extrap_drop = (double)value * 1e-6;
    } else if (k == "symmetry") {
        if (value < 0 || value > 1) return fail(KS_ERR_ARG, "symmetry must be 0 (none) or 1 (Xi)");
        h->xi = (int)value;
    } else if (k == "stall_window") {
        if (value < 1) return fail(KS_ERR_ARG, "stall_window must be >= 1");
        h->stall_window = value;
    } else if (k == "stall_drop_ppm") {
        if (value < 0 || value >= 1000000) return fail(KS_ERR_ARG, "stall_drop_ppm in [0, 1e6)");
        h->stall_drop = (double)value * 1e-6;
    } else if (k == "graph") {
        h->graph = value ? 1 : 0;
    } else if (k == "row_threads" || k == "col_threads") {
        if (value != 128 && value != 256) return fail(KS_ERR_ARG, k + " must be 128 or 256");
        for (int pr = 0; pr < 2; ++pr) (k == "row_threads" ? h->lrow : h->lcol)[pr].threads = (int)value;
        drop_graphs(h);
    } else if (k == "chunk") {
        if (value < 1) return fail(KS_ERR_ARG, "chunk must be >= 1");
        h->chunk = (int)std::min<long long>(value, 1 << 30);
    } else {
        return fail(KS_ERR_ARG, "unknown option " + k);
    }
    return KS_OK;
}

extern "C" int ks_get_option(ks_loop_t h, const char* key, long long* value) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!key || !value) return fail(KS_ERR_ARG, "null argument");
    const std::string k(key);
    if (k == "path") *value = h->path[h->mode == KS_FP64 ? P64 : P32];
    else if (k == "path_f64") *value = h->path[P64];
    else if (k == "path_f32") *value = h->path[P32];
    else if (k == "cluster_f64") *value = h->cplan[0].bytes ? h->cplan[0].C : 0;
    else if (k == "cluster_f32") *value = h->cplan[1].bytes ? h->cplan[1].C : 0;
    else if (k == "cluster_smem_f64") *value = h->cplan[0].bytes;
    else if (k == "cluster_exchange") *value = h->cexchange;
    else if (k == "cluster_grid_f64") *value = h->cplan[0].bytes ? h->cgrid[0] : 0;
    else if (k == "cluster_min_blocks_f64") *value = h->cplan[0].bytes ? h->cplan[0].mb : 0;
    else if (k == "cluster_min_blocks_f32") *value = h->cplan[1].bytes ? h->cplan[1].mb : 0;
    else if (k == "cluster_grid_f32") *value = h->cplan[1].bytes ? h->cgrid[1] : 0;
    else if (k == "cluster_exchange_f64") *value = h->cplan[0].bytes ? h->cplan[0].ax : 0;
    else if (k == "cluster_exchange_f32") *value = h->cplan[1].bytes ? h->cplan[1].ax : 0;
    else if (k == "cluster_smem_f32") *value = h->cplan[1].bytes;
    else if (k == "rows_per_tile") *value = h->rows_per_tile;
    else if (k == "finish_f32_adjoint") *value = h->finish_f32_adjoint;
    else if (k == "switch_probe") *value = h->switch_probe;
    else if (k == "switch_probe_steps") *value = h->probe_steps;
    else if (k == "cluster_threads") *value = h->cthreads;
    else if (k == "cluster_block_f64") *value = h->cplan[0].bytes ? cluster_block(h, 0, h->cplan[0]) : 0;
    else if (k == "cluster_block_f32") *value = h->cplan[1].bytes ? cluster_block(h, 1, h->cplan[1]) : 0;
    else if (k == "cluster_block_mixed_finish") *value = h->cplan[2].bytes ? cluster_block(h, 2, h->cplan[2]) : 0;
    else if (k == "cluster_mixed_finish") *value = h->cplan[2].bytes ? h->cplan[2].C : 0;
    else if (k == "stall_window") *value = h->stall_window;
    else if (k == "stall_drop_ppm") *value = std::llround(h->stall_drop * 1e6);
    else if (k == "chunk") *value = h->chunk;
    else if (k == "graph") *value = h->graph;
    else if (k == "row_threads") *value = h->lrow[P64].threads;
    else if (k == "col_threads") *value = h->lcol[P64].threads;
    else if (k == "graph_replays") *value = h->graph_replays;
    else if (k == "symmetry") *value = h->xi;
    else if (k == "extrapolate") *value = h->extrapolate;
    else if (k == "extrapolate_start_ppm") *value = std::llround(h->extrap_start * 1e6);
    else if (k == "extrapolate_drop_ppm") *value = std::llround(h->extrap_drop * 1e6);
    else if (k == "extrapolations") *value = h->n_extrap;
    else if (k == "extrapolations_rejected") *value = h->n_extrap_rejected;
    else return fail(KS_ERR_ARG, "unknown option " + k);
    return KS_OK;
}

extern "C" int ks_get_history(ks_loop_t h, int b, long long* steps, double* sqrtJ, int* prec,
                              int cap) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (b < 0 || b >= h->d.B) return fail(KS_ERR_ARG, "loop index out of range");
    if (b >= (int)h->hist_steps.size()) return 0;
    const int n = (int)h->hist_steps[b].size();
    for (int i = 0; i < n && i < cap; ++i) {
        if (steps) steps[i] = h->hist_steps[b][i];
        if (sqrtJ) sqrtJ[i] = h->hist_sqrtJ[b][i];
        if (prec) prec[i] = h->hist_prec[b][i];
    }
    return n;
}

// ------------------------------------------------------------------------------------------
// Autotuner: time the launch candidates of this batch on a synthetic band-limited state and
// keep the fastest.  Candidates: the cluster-resident kernel for every cluster size whose
// shared-memory plan fits, with 128 or 256 threads per CTA; the grid-persistent kernel; four
// launches per step.  The tuned precision is the one a descent spends its bulk in (float for
// KS_FP32 and KS_MIXED handles, double for KS_FP64).  Choices are cached in the text file named
// by the environment variable KS_AUTOTUNE_CACHE, if set, keyed by the batch shape and mode.
// ------------------------------------------------------------------------------------------
namespace {

struct TuneChoice {
    int path, cluster, threads;
};

std::string tune_key(const ks_loop* h) {
    unsigned long long hs = 1469598103934665603ull;  // FNV-1a over the Ns list
    for (int v : h->ns) {
        hs ^= (unsigned long long)v;
        hs *= 1099511628211ull;
    }
    char buf[160];
    std::snprintf(buf, sizeof(buf), "nx=%d B=%d ns=%016llx mode=%d scheme=%d", h->d.nx, h->d.B, hs,
                  h->mode, h->d.scheme);
    return buf;
}

bool cache_lookup(const std::string& key, TuneChoice& c) {
    const char* path = std::getenv("KS_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[256];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        std::string ln(line);
        const size_t bar = ln.find('|');
        if (bar == std::string::npos || ln.substr(0, bar) != key) continue;
        TuneChoice t{};
        // only the launch shapes the tuner itself tries (the cluster kernel needs 128 or 256
        // threads: its phase B' splits the block into the last warp and the rest)
        if (std::sscanf(ln.c_str() + bar + 1, "%d %d %d", &t.path, &t.cluster, &t.threads) == 3 &&
            t.path >= 0 && t.path <= 2 && t.cluster >= 0 && t.cluster <= 16 &&
            (t.threads == 128 || t.threads == 256)) {
            c = t;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(const std::string& key, const TuneChoice& c) {
    const char* path = std::getenv("KS_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s|%d %d %d\n", key.c_str(), c.path, c.cluster, c.threads);
    std::fclose(f);
}

// the tuned precision's launch form (both for single-precision handles; the float bulk of a
// KS_MIXED handle, whose double finish keeps the default rule's form)
int apply_choice(ks_loop* h, const TuneChoice& c) {
    h->path[P32] = c.path;
    if (h->mode != KS_MIXED) h->path[P64] = c.path;
    h->force_cluster = c.cluster;
    h->cthreads = c.threads;
    KS_TRY((setup_cluster<double, double>(h)));
    KS_TRY((setup_cluster<float, float>(h)));
    if (h->mode == KS_MIXED) KS_TRY((setup_cluster<double, float>(h)));
    return KS_OK;
}

}  // namespace

int ks_autotune_impl(ks_loop* h) {
    const std::string key = tune_key(h);
    TuneChoice best{0, 0, 128};
    if (cache_lookup(key, best)) return apply_choice(h, best);
    const int pr = (h->mode == KS_FP64) ? P64 : P32;
    // synthetic state: a few band modes of amplitude ~0.5, T = 40, on the grid (double)
    const int nx = h->d.nx;
    std::vector<double> u((size_t)h->ngrid);
    for (int b = 0; b < h->d.B; ++b) {
        const int ns = h->ns[b];
        for (int n = 0; n < ns; ++n)
            for (int m = 0; m < nx; ++m) {
                const double x = 6.283185307179586 * m / nx, t = 6.283185307179586 * n / ns;
                u[(size_t)h->goff[b] + (size_t)n * nx + m] =
                    0.5 * std::sin(x + t) + 0.3 * std::cos(2 * x - t) + 0.1 * std::sin(3 * x + 2 * t);
            }
    }
    std::vector<double> T(h->d.B, 40.0);
    std::vector<float> uf;
    const void* usrc = u.data();
    if (h->mode == KS_FP32) {
        uf.assign(u.begin(), u.end());
        usrc = uf.data();
    }
    double* dT = nullptr;
    void* du = nullptr;
    KS_TRY(dev_alloc(h, (void**)&dT, h->d.B * sizeof(double)));
    KS_TRY(dev_alloc(h, &du, (size_t)h->ngrid * elem_size(h->mode == KS_FP32 ? P32 : P64)));
    KS_CUDA(cudaMemcpy(dT, T.data(), h->d.B * sizeof(double), cudaMemcpyHostToDevice));
    KS_CUDA(cudaMemcpy(du, usrc, (size_t)h->ngrid * elem_size(h->mode == KS_FP32 ? P32 : P64),
                       cudaMemcpyHostToDevice));
    std::vector<TuneChoice> cands;
    for (int C : {16, 8, 4, 2, 1})
        for (int th : {128, 256}) cands.push_back(TuneChoice{0, C, th});
    cands.push_back(TuneChoice{1, 0, 128});
    cands.push_back(TuneChoice{2, 0, 128});
    cudaEvent_t e0, e1;
    KS_CUDA(cudaEventCreate(&e0));
    KS_CUDA(cudaEventCreate(&e1));
    const int S = std::max(2, (int)std::min<long long>(40, 4000000LL / std::max<long long>(1, h->ngrid)));
    float best_ms = 1e30f;
    for (const TuneChoice& c : cands) {
        if (apply_choice(h, c) != KS_OK) continue;
        if (c.path == 0) {
            const int slot = pr == P64 ? 0 : 1;
            if (!h->cplan[slot].bytes || h->cplan[slot].C != c.cluster) continue;
        }
        if (c.path == 1 && !h->pgrid[pr]) continue;
        if (set_state_full(h, du, dT, 0) != KS_OK) continue;
        if (steps_impl(h, 2, 0.0, 0) != KS_OK) continue;
        KS_CUDA(cudaEventRecord(e0, 0));
        for (int rep = 0; rep < 3; ++rep)
            if (steps_impl(h, S, 0.0, 0) != KS_OK) break;
        KS_CUDA(cudaEventRecord(e1, 0));
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->state_set = false;
    h->launches = 0;
    cache_store(key, best);
    return apply_choice(h, best);
}

extern "C" int ks_autotune(ks_loop_t h) {
    g_err.clear();
    KS_TRY(check_handle(h));
    KS_TRY(ks_autotune_impl(h));
    KS_CUDA(cudaDeviceSynchronize());
    return KS_OK;
}

// ------------------------------------------------------------------------------------------
// Band-level state I/O (bitwise checkpoints): the band of every loop as interleaved complex
// doubles, loops in batch order, each [j][k + Ks] with j = 0..Kx, k = -Ks..Ks.
// ------------------------------------------------------------------------------------------
namespace {
__global__ void k_band_d2f_sel(const cpx<double>* src, cpx<float>* dst, const long long* boff,
                               const int* prec, int B, int nkx, const int* ks) {
    const int b = blockIdx.y;
    if (b >= B || prec[b] != 1) return;
    const long long n = (long long)nkx * (2 * ks[b] + 1);
    const long long o = boff[b];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[o + i] = mk<float>((float)src[o + i].x, (float)src[o + i].y);
}
}  // namespace

extern "C" long long ks_band_size(ks_loop_t h) { return h ? h->nband : -1; }

extern "C" int ks_get_band(ks_loop_t h, double* band, double* T, int* prec, long long* steps,
                           void* stream) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!h->state_set) return fail(KS_ERR_STATE, "ks_get_band before ks_set_state");
    cudaStream_t s = (cudaStream_t)stream;
    KS_TRY(readback(h, s));
    Work& w = h->st;
    Work& a = h->api;
    const int B = h->d.B;
    if (h->need[P32]) {
        dim3 g(8, B);
        k_band_merge<<<g, 256, 0, s>>>((const cpx<float>*)w.uh[P32], (const cpx<double>*)w.uh[P64],
                                       (cpx<double>*)a.uh[P64], h->d_boff, w.prec, B, h->d.nkx, h->d_ks);
        KS_CUDA(cudaGetLastError());
    } else {
        KS_CUDA(cudaMemcpyAsync(a.uh[P64], w.uh[P64], (size_t)h->nband * sizeof(cpx<double>),
                                cudaMemcpyDeviceToDevice, s));
    }
    KS_TRY(copy_out(band, a.uh[P64], (size_t)h->nband * sizeof(cpx<double>), s));
    KS_TRY(copy_out(T, w.T + (size_t)w.par * B, B * sizeof(double), s));
    KS_TRY(copy_out(steps, w.steps, B * sizeof(long long), s));
    if (prec) KS_CUDA(cudaMemcpyAsync(prec, h->h_prec.data(), B * sizeof(int), cudaMemcpyDefault, s));
    KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}

extern "C" int ks_set_band(ks_loop_t h, const double* band, const double* T, const int* prec,
                           const long long* steps, void* stream) {
    g_err.clear();
    KS_TRY(check_handle(h));
    if (!band || !T) return fail(KS_ERR_ARG, "band and T are required");
    cudaStream_t s = (cudaStream_t)stream;
    Work& w = h->st;
    const int B = h->d.B;
    std::vector<int> pv(B, start_prec(h));
    if (prec) {
        KS_CUDA(cudaMemcpy(pv.data(), prec, B * sizeof(int), cudaMemcpyDefault));
        for (int b = 0; b < B; ++b) {
            if (pv[b] != P64 && pv[b] != P32) return fail(KS_ERR_ARG, "precision must be 0 or 1");
            if (!h->need[pv[b]]) return fail(KS_ERR_ARG, "precision not available in this mode");
        }
    }
    KS_CUDA(cudaMemcpyAsync(w.uh[P64], band, (size_t)h->nband * sizeof(cpx<double>), cudaMemcpyDefault, s));
    KS_CUDA(cudaMemcpyAsync(w.T, T, B * sizeof(double), cudaMemcpyDefault, s));
    w.par = 0;
    k_prep_wT<<<(B + 127) / 128, 128, 0, s>>>(w.T, w.wT, B);
    KS_CUDA(cudaGetLastError());
    h->h_prec = pv;
    KS_CUDA(cudaMemcpyAsync(w.prec, h->h_prec.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    if (h->need[P32]) {
        dim3 g(8, B);
        k_band_d2f_sel<<<g, 256, 0, s>>>((const cpx<double>*)w.uh[P64], (cpx<float>*)w.uh[P32], h->d_boff,
                                         w.prec, B, h->d.nkx, h->d_ks);
        KS_CUDA(cudaGetLastError());
    }
    KS_CUDA(cudaMemsetAsync(w.status, 0, B * sizeof(int), s));
    KS_CUDA(cudaMemsetAsync(w.sqrtJ, 0, B * sizeof(double), s));
    if (steps) KS_CUDA(cudaMemcpyAsync(w.steps, steps, B * sizeof(long long), cudaMemcpyDefault, s));
    else KS_CUDA(cudaMemsetAsync(w.steps, 0, B * sizeof(long long), s));
    h->h_status.assign(B, KS_RUNNING);
    w.mix_valid[P64] = w.mix_valid[P32] = false;
    h->state_set = true;
    h->hist_steps.assign(B, {});
    h->hist_sqrtJ.assign(B, {});
    h->hist_prec.assign(B, {});
    KS_CUDA(cudaStreamSynchronize(s));
    return KS_OK;
}
