// ks_cluster.cuh - cluster-resident tau-descent: one thread-block cluster per loop.
//
// A loop's whole working set lives in the distributed shared memory of one cluster of C CTAs
// (1 <= C <= 16) for a chunk of tau-steps:
//   * column j (retained x-mode, 0..Kx) is owned by rank j % C, slot j / C: its band values
//     u_hat, r_hat and its mixed-array column M[j][n] (n = 0..Ns-1) sit in that rank's SMEM.  In
//     the centre-symmetric subspace (p.xi) the columns go by pairs (2p + 1, 2p + 2): pair p is
//     owned by rank p % C, slots 2 (p / C) and 2 (p / C) + 1, and each pair shares one complex
//     s-transform (see col_pair_item in ks_items.cuh); column 0 is zero and owned by no rank;
//   * rows n are split in contiguous blocks of an even number of rows per rank; a rank keeps
//     the grid values of u for its rows between the two row phases (in SMEM, or in the global
//     U array when the plan cannot hold them).
// The four phases of a tau-step (see ks_items.cuh) exchange data through DSMEM: a row phase
// gathers the columns' values for its rows from the owners and scatters its results back.
// Each exchange is a set of asynchronous remote stores (st.async) that count their bytes on an
// mbarrier of the receiving CTA; a CTA starts its next phase once the bytes it expects have
// landed (plans without room for the second column buffer this needs, and the knob
// "cluster_exchange" = 0, separate the phases by hardware cluster barriers instead).  There is
// no grid-wide synchronisation and no global-memory round trip inside a step.  Column owners broadcast their partials of
// J and L^dag_2 to every rank; every rank sums them in the same fixed order, so all ranks
// take the same freeze decision and advance T identically.  The per-element arithmetic and
// the reduction orders are those of the per-phase items, so results agree bit for bit.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "ks_items.cuh"

namespace ks {

namespace cgx = cooperative_groups;

// Shared-memory plan of one cluster launch (byte offsets into the dynamic shared memory).
struct ClusterPlan {
    int C;        // cluster size
    int rt;       // largest row batch of one x-transform call (even power of two)
    int ncmax;    // max columns per rank
    int nsmax;    // max Ns over the batch
    int nkmax;    // max 2 Ks + 1
    int rmax;     // max rows per rank
    int off_M, off_uh, off_rh, off_U, off_scr, off_part, off_red, off_tw, off_rin, off_tw_a;
    int off_tab;  // per-x-mode tables q_j, q_j^2 - q_j^4, q_j^4 (q_j^2 - 1)^2 (and the second in RA)
    int bytes;
    int u_global;  // 1: the rank's grid rows of u live in global memory (U array), not SMEM
    // mbarrier exchanges (ax = 1): a second column buffer (off_M2) receives the phase-A' results,
    // so that no exchange writes a buffer its receiver may still be reading (see k_cluster), and
    // four mbarriers (off_bar), one per exchange of a step.  ax = 0: off_M2 = off_M, cluster
    // barriers.
    int ax, off_M2, off_bar;
    int* err;      // set to 1 when an exchange wait gives up (bounded, see xbar_wait)
    int mb;        // the kernel's minimum resident blocks per SM (launch bounds): 1 or 2
};

// ---- mbarrier exchanges ---------------------------------------------------------------------
// A producer writes its values into the receiver's shared memory with st.async, each store
// counting its bytes (complete_tx) on the receiver's mbarrier of that exchange; the receiver
// arms the barrier with the byte count it expects (one arrival, arrive.expect_tx) and waits for
// the phase to complete.  Stores may land before the arming: the transaction count then runs
// negative until it.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// shared::cluster address of the same offset in the shared memory of cluster rank `rank`
__device__ __forceinline__ unsigned cluster_u32(unsigned a, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void xbar_init(unsigned bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void xbar_arm(unsigned bar, unsigned bytes) {
    unsigned long long state;
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state) : "r"(bar), "r"(bytes) : "memory");
    (void)state;
}

__device__ __forceinline__ bool xbar_test(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long xbar_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of parity `parity`; true once it completed.  Bounded: after about a second
// of the global timer (or 2^26 polls) the wait gives up, sets *err and returns false, and it
// returns false at once when another wait has set *err.  The caller then stops arming and
// pushing (k_cluster: xdead), so the launch runs out its steps without waiting and the host
// reports the error; every thread takes the same path through the kernel's block barriers.
__device__ __forceinline__ bool xbar_wait(unsigned bar, unsigned parity, int* err) {
    if (xbar_test(bar, parity)) return true;
    const unsigned long long t0 = xbar_clock_ns();
    for (unsigned it = 1;; ++it) {
        if (xbar_test(bar, parity)) return true;
        if ((it & 15) == 0) {
            if (*(volatile int*)err) return false;
            if (it > (1u << 26) || xbar_clock_ns() - t0 > 1000000000ull) {
                atomicExch(err, 1);
                return false;
            }
        }
    }
}

// Two adjacent complex values to shared::cluster address dst (16-byte aligned), counted on bar.
__device__ __forceinline__ void st_async_pair(unsigned dst, cpx<float> a, cpx<float> b, unsigned bar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];"
        ::"r"(dst), "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "r"(bar) : "memory");
}
__device__ __forceinline__ void st_async_pair(unsigned dst, cpx<double> a, cpx<double> b, unsigned bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
                 ::"r"(dst), "d"(a.x), "d"(a.y), "r"(bar) : "memory");
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];"
                 ::"r"(dst + 16u), "d"(b.x), "d"(b.y), "r"(bar) : "memory");
}
// One partial (8 bytes, 8-byte aligned).
__device__ __forceinline__ void st_async_part(unsigned dst, double v, unsigned bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];"
                 ::"r"(dst), "d"(v), "r"(bar) : "memory");
}
__device__ __forceinline__ void st_async_part(unsigned dst, ff v, unsigned bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];"
                 ::"r"(dst), "f"(v.hi), "f"(v.lo), "r"(bar) : "memory");
}

// rows per rank: an even number covering Ns with C ranks
__host__ __device__ inline int cluster_rows_per_rank(int ns, int C) {
    int r = (ns + C - 1) / C;
    r += (r & 1);
    return r < 2 ? 2 : r;
}

// FFT of `cnt` columns stored [q][n] at `a` with `b` as scratch; the result is left in `a`.
// nthr > 0: a double transform run by the first nthr threads only (see fft_batch), which alone
// call this; otherwise every thread of the block calls it.
template <typename R>
__device__ __forceinline__ void col_fft_inplace(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir,
                                                const cpx<R>* tw, int nthr = 0) {
    cpx<R>* r = nthr > 0 ? fft_col<R, true>(a, b, lg, cnt, dir, tw, nthr)
                         : fft_col_warp<R, true>(a, b, lg, cnt, dir, tw);
    if (r != a) {
        const int n = cnt << lg;
        const int NT = nthr > 0 ? nthr : (int)blockDim.x;
        for (int i = threadIdx.x; i < n; i += NT) a[i] = r[i];
        if (nthr > 0) part_sync(nthr);
        else __syncthreads();
    }
}

// Two adjacent complex values to (possibly remote) shared memory: one 16-byte store for float
// (the address is 16-byte aligned at every call site: even element index, aligned base), two
// for double.  Halves the DSMEM store transactions of the float exchange.
template <typename X>
__device__ __forceinline__ void store_pair(cpx<X>* dst, cpx<X> a, cpx<X> b) {
    if constexpr (sizeof(X) == 4) {
        *reinterpret_cast<float4*>(dst) = make_float4(a.x, a.y, b.x, b.y);
    } else {
        dst[0] = a;
        dst[1] = b;
    }
}

// Tables in the precision of the adjoint half of a step (twiddles, q_j, q_j^2 - q_j^4).
template <typename RA>
struct AdjTables {
    const cpx<RA>* tw;
    const RA* qv;
    const RA* lin;
};

// R: precision of the state, the residual half of a step (phases A, B), the reductions and the
// update.  RA: precision of the adjoint half (the inverse transform of i q r_hat, phase A' and
// the forward transform and G_hat assembly of phase B').  RA = R is the plain float or double
// descent; R = double, RA = float is the finishing stage of a mixed descent, where r, J,
// dJ/dT and the update stay in double and only the descent direction is formed in float.
// Launch bounds: up to 256 threads and MB resident blocks per SM.  MB = 1 leaves ptxas its
// choice (128-157 registers, no spills; with the thread bound alone it held the double kernel
// to 64 registers and spilled), the faster form for one loop; MB = 2 caps it at 128 (it then
// takes 96-113, no spills), which lets three blocks of 160 threads share an SM (a sub-partition
// holds four warps of at most 128 registers), so a batch of 16 loops in clusters of 16 runs in
// one wave instead of two (batch16_64x64: 17.3 -> 10.7 us float, 48.9 -> 29.4 us double, while
// one 64x128 loop takes 9.14 -> 9.46 and 28.5 -> 28.8 us).  The plan picks MB by occupancy
// (setup_cluster).
// XI: the centre-symmetric subspace (p.xi set), a separate instantiation so that each kernel
// carries only the code of its own column scheme.
template <typename R, typename RA, bool XI, int MB>
__global__ void __launch_bounds__(256, MB) k_cluster(Dims d, Bufs<R> p, AdjTables<RA> ta,
                                                 ClusterPlan cp, int nsteps, int par0, int use_M) {
    typedef typename PartT<R>::type Part;
    constexpr bool kSame = sizeof(R) == sizeof(RA);
    extern __shared__ __align__(16) unsigned char smem[];
    cgx::cluster_group cl = cgx::this_cluster();
    const int C = cp.C;
    const int rank = (int)cl.block_rank();
    const int cid = blockIdx.x / C;
    const int ncl = gridDim.x / C;
    const int tid = threadIdx.x, nt = blockDim.x;
    // A block of 4k + 1 warps (see cluster_block) carries one extra warp, which forms the
    // scalars of a step (step_scalars) beside the work of the other 4k warps (ntw threads).  The
    // element loops of a step run on the work warps only and the extra warp starts them past
    // their end (wtid); a double transform of such a plan has at most ntw butterflies a pass, so
    // the extra warp gets none there either.
    const int ntw = nt - (nt % 64);
    const int wtid = (tid < ntw) ? tid : (1 << 30);
    const bool xw = ntw != nt;     // the block has the extra warp
    // Where the extra warp forms the scalars: in phase A' for a float state (there its double
    // arithmetic finds the FP64 pipe idle; in phase B' it held up the whole phase, 3.7 k of the
    // 22.7 k clocks of the 64x128 float step), in phase B' for a double state (beside the
    // s-transform of w_hat, which hides it; in phase A' it takes the FP64 pipe from the work
    // warps, measured 1 % slower).
    const bool sa = xw && sizeof(R) == 4;
    const int wn = sa ? ntw : 0;   // thread count of the phase-A' transforms (0: the block)
    auto wsync = [&]() {           // barrier of the threads that run phase A'
        if (sa) part_sync(ntw);
        else __syncthreads();
    };
    const int nx = d.nx, lgnx = d.lgnx, kx = d.kx, nkx = d.nkx, B = d.B;
    const int rmax = cp.rmax;
    constexpr bool xi = XI;
    // owner rank and slot of x-mode j (j >= 1 in the subspace)
    auto own_rank = [&](int j) { return xi ? ((j - 1) >> 1) % C : j % C; };
    auto own_slot = [&](int j) { return xi ? 2 * (((j - 1) >> 1) / C) + ((j - 1) & 1) : j / C; };
    cpx<R>* Mloc = reinterpret_cast<cpx<R>*>(smem + cp.off_M);   // owned columns: P / W
    cpx<R>* Rin = reinterpret_cast<cpx<R>*>(smem + cp.off_rin);  // own rows: v / rho, [j][r]
    cpx<R>* uhl = reinterpret_cast<cpx<R>*>(smem + cp.off_uh);
    cpx<R>* rhl = reinterpret_cast<cpx<R>*>(smem + cp.off_rh);
    R* const Us = reinterpret_cast<R*>(smem + cp.off_U);  // rows of u kept between row phases
    cpx<R>* scr = reinterpret_cast<cpx<R>*>(smem + cp.off_scr);
    Part* part = reinterpret_cast<Part*>(smem + cp.off_part);  // [2][nkx]: J, L2 partials
    double* red = reinterpret_cast<double*>(smem + cp.off_red);
    cpx<R>* tws = reinterpret_cast<cpx<R>*>(smem + cp.off_tw);
    // adjoint-precision views of the same buffers (phases are separated by barriers)
    cpx<RA>* Rin_a = reinterpret_cast<cpx<RA>*>(Rin);
    cpx<RA>* Mloc_a = reinterpret_cast<cpx<RA>*>(Mloc);
    // mbarrier exchanges (ax): the phase-A' results land in a second column buffer, which phase
    // B' also works in, so Mloc is only ever written by phase A's exchange and read in phase B
    cpx<R>* const Mloc2 = reinterpret_cast<cpx<R>*>(smem + cp.off_M2);
    cpx<RA>* const Mloc2_a = reinterpret_cast<cpx<RA>*>(Mloc2);
    const bool ax = cp.ax != 0;
    const unsigned xbar0 = smem_u32(smem + cp.off_bar);  // exchange x: xbar0 + 8 x
    unsigned xpar = 0;  // bit x: parity of the next phase of exchange x's mbarrier
    bool xdead = false;  // a wait of this thread gave up: no more arming, pushing or waiting
    cpx<RA>* scr_a = reinterpret_cast<cpx<RA>*>(scr);
    cpx<RA>* tws_a = kSame ? reinterpret_cast<cpx<RA>*>(tws) : reinterpret_cast<cpx<RA>*>(smem + cp.off_tw_a);
    // 1/(2 Nx) of the row split; per loop it is multiplied by 1/Ns, the normalisation of the
    // forward s-transform that the column phases would otherwise apply (both powers of two, so
    // the product is exact and scaling before the transform gives the same bits as after it)
    const R h0 = (R)d.hx;
    const RA h0_a = (RA)d.hx;
    // the per-x-mode tables, read in every phase, live in shared memory
    R* const s_qv = reinterpret_cast<R*>(smem + cp.off_tab);
    R* const s_lin = s_qv + nkx;
    R* const s_cq = s_lin + nkx;
    RA* const s_lina = reinterpret_cast<RA*>(s_cq + nkx);
    // Start-up: the per-mode tables and the twiddles the launch's transforms read are copied
    // with asynchronous copies (cp_async), which the threads do not wait for; the loop's state
    // follows the same way, so all of them share one round trip to memory.  They are waited
    // for before the barrier that closes the state load; the tables are first read after it.
    // A launch of one loop (B = 1) needs no load to find it: index 0, offsets 0, Ns = nsmax.
    const bool one = (B == 1);
    const int b_first = (!one && cid < B) ? p.colorder[cid] : 0;
    for (int i = tid; i < nkx; i += nt) {
        cp_async<sizeof(R)>(s_qv + i, p.qv + i);
        cp_async<sizeof(R)>(s_lin + i, p.lin + i);
        cp_async<sizeof(R)>(s_cq + i, p.cq + i);
        cp_async<sizeof(RA)>(s_lina + i, ta.lin + i);
    }
    if (xi && tid == 0) {  // column 0 is zero in the subspace and owned by no rank
        part[0] = Part{};
        part[nkx] = Part{};
    }
    const int nm = max(nx, cp.nsmax);  // longest transform of the launch
    load_twiddles(tws, p.tw, nm);
    if (!kSame) load_twiddles(tws_a, ta.tw, nm);
    if (ax && tid == 0) {
        // first used after the cluster barrier that precedes a loop's steps
        for (int x = 0; x < 4; ++x) xbar_init(xbar0 + 8u * x);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    for (int bi = cid; bi < B; bi += ncl) {
        const int b = one ? 0 : ((bi == cid) ? b_first : p.colorder[bi]);
        // the skip test and the per-loop scalars in one round of loads; every rank reads the
        // same global words, so the skip is uniform across the cluster
        const int prec_b = p.prec[b], status_b = p.status[b];
        const int ns = one ? cp.nsmax : p.ns[b];
        const int lg = one ? __ffs(cp.nsmax) - 1 : p.lgns[b];
        const int ks = one ? cp.nsmax / 3 : p.ks[b];
        const int nk = 2 * ks + 1;
        const R ins = p.insv[b];
        const R h = h0 * ins;
        const RA h_a = h0_a * (RA)ins;
        const size_t bo = one ? 0 : (size_t)p.boff[b];
        const long long moff_b = one ? 0 : p.moff[b], goff_b = one ? 0 : p.goff[b];
        double T = p.T[(size_t)par0 * B + b];
        double wT = p.wT[(size_t)par0 * B + b];
        // local column q <-> x-mode j (in the subspace by pairs; a second column past Kx is a
        // ghost that holds zeros and is never stored)
        const int npr = (kx + 1) >> 1;
        const int ncol = xi ? ((rank < npr) ? 2 * ((npr - rank + C - 1) / C) : 0)
                            : ((rank < nkx) ? (nkx - rank + C - 1) / C : 0);
        auto colj = [&](int q) { return xi ? 2 * (rank + (q >> 1) * C) + 1 + (q & 1) : rank + q * C; };
        const int rpr = cluster_rows_per_rank(ns, C);
        const int row0 = rank * rpr;
        const int nrow = (row0 < ns) ? min(rpr, ns - row0) : 0;
        cpx<R>* Mg = p.M + moff_b;
        // bytes each exchange of a step delivers to this rank: phase A (A'), the values of its
        // real columns at every row; phase B, the values of its rows in every exchanged column
        // and two partials per column; phase B', the values of its rows in every column
        int mycols = ncol;
        if (xi) {
            mycols = 0;
            for (int q = 0; q < ncol; ++q) mycols += (colj(q) <= kx) ? 1 : 0;
        }
        const int ncx = xi ? kx : nkx;
        const unsigned bx_A = (unsigned)(mycols * ns) * (unsigned)sizeof(cpx<R>);
        const unsigned bx_B = (unsigned)(ncx * nrow) * (unsigned)sizeof(cpx<RA>) + 2u * ncx * (unsigned)sizeof(Part);
        const unsigned bx_Aa = (unsigned)(mycols * ns) * (unsigned)sizeof(cpx<RA>);
        const unsigned bx_Ba = (unsigned)(ncx * nrow) * (unsigned)sizeof(cpx<R>);
        R* Ul = cp.u_global ? p.U + goff_b + (size_t)row0 * nx : Us;

        // ---- the band of the owned columns, and the rows' mixed values (when valid) ----
        auto load_state = [&]() {
            for (int i = tid; i < ncol * nk; i += nt) {
                const int q = i / nk, kk = i - q * nk;
                const int j = colj(q);
                if (j <= kx) cp_async<sizeof(cpx<R>)>(uhl + i, p.uh + bo + (size_t)j * nk + kk);
                else uhl[i] = mk<R>(0, 0);
            }
            if (use_M) {
                for (int i = tid; i < nkx * nrow; i += nt) {
                    const int j = i / nrow, r = i - j * nrow;
                    if (xi && j == 0) Rin[r] = mk<R>(0, 0);  // the zero column of the subspace
                    else cp_async<sizeof(cpx<R>)>(Rin + (size_t)j * rmax + r, Mg + (size_t)j * ns + row0 + r);
                }
            } else if (xi) {
                for (int r = tid; r < nrow; r += nt) Rin[r] = mk<R>(0, 0);
            }
        };
        if (one) load_state();  // its addresses need no load: issued with the scalars
        if (prec_b != p.myprec || status_b != ST_RUNNING) {
            if (rank == 0 && tid == 0 && status_b != ST_RUNNING &&
                (prec_b == p.myprec || !p.own_frozen_only)) {
                p.T[(size_t)(par0 ^ 1) * B + b] = T;
                p.wT[(size_t)(par0 ^ 1) * B + b] = wT;
            }
            cp_async_wait();  // no copy may land in shared memory the next loop reuses
            continue;
        }
        if (!one) load_state();

        // two adjacent values to the same offset (local pointer `local`) in the shared memory of
        // rank rk: counted on rk's mbarrier of exchange x (x >= 0 and ax), or plain DSMEM stores
        auto xput = [&](auto* local, int rk, int x, auto a, auto b) {
            if (ax && x >= 0) {
                if (!xdead) st_async_pair(cluster_u32(smem_u32(local), rk), a, b, cluster_u32(xbar0 + 8u * x, rk));
            } else {
                store_pair(cl.map_shared_rank(local, rk), a, b);
            }
        };
        // partial slot j of rank rk (exchange 1, phase B)
        auto xpart = [&](int j, int rk, Part v) {
            if (ax) {
                if (!xdead) st_async_part(cluster_u32(smem_u32(part + j), rk), v, cluster_u32(xbar0 + 8u, rk));
            } else {
                cl.map_shared_rank(part, rk)[j] = v;
            }
        };
        // push a column result X[q][n] (n = 0..Ns-1) to the row owners' Rin[j][n - row0(owner)],
        // two rows per store (rows per rank and rmax are even, so a pair has one owner)
        auto push_columns = [&](const auto* X, auto* RinT, int x) {
            for (int i = wtid; i < (ncol << lg) >> 1; i += ntw) {
                const int q = (2 * i) >> lg, n = (2 * i) & (ns - 1);
                const int owner = n / rpr;
                xput(RinT + (size_t)colj(q) * rmax + (n - owner * rpr), owner, x, X[2 * i], X[2 * i + 1]);
            }
        };
        // push the s-inverse c of each column pair: column 2p+1 gets Re c, column 2p+2 Im c, as
        // the imaginary parts (imag = true: u, v) or the real parts (rho)
        auto push_pairs = [&](const auto* Cp, auto* RinT, bool imag, int x) {
            typedef typename std::remove_pointer<decltype(RinT)>::type CT;
            typedef decltype(CT{}.x) X;
            for (int i = wtid; i < (ncol << lg) >> 2; i += ntw) {
                const int pp = (2 * i) >> lg, n = (2 * i) & (ns - 1);
                const int owner = n / rpr;
                auto* dst = RinT + (n - owner * rpr);
                const auto c0 = Cp[2 * i], c1 = Cp[2 * i + 1];
                const int ja = colj(2 * pp), jb = ja + 1;
                if (imag) xput(dst + (size_t)ja * rmax, owner, x, mk<X>(0, c0.x), mk<X>(0, c1.x));
                else xput(dst + (size_t)ja * rmax, owner, x, mk<X>(c0.x, 0), mk<X>(c1.x, 0));
                if (jb <= kx) {
                    if (imag) xput(dst + (size_t)jb * rmax, owner, x, mk<X>(0, c0.y), mk<X>(0, c1.y));
                    else xput(dst + (size_t)jb * rmax, owner, x, mk<X>(c0.y, 0), mk<X>(c1.y, 0));
                }
            }
        };

        cp_async_wait();
        __syncthreads();
        if (!use_M) {
            // no valid mixed values: prime them from the band (s-inverse of the owned columns)
            if (xi) {
                for (int i = wtid; i < (ncol >> 1) << lg; i += ntw) {
                    const int pp = i >> lg, n = i & (ns - 1);
                    const int k = (n < (ns >> 1)) ? n : n - ns;
                    Mloc[i] = (k >= -ks && k <= ks)
                                  ? xi_join_imag(uhl[(2 * pp) * nk + k + ks], uhl[(2 * pp + 1) * nk + k + ks])
                                  : mk<R>(0, 0);
                }
                __syncthreads();
                col_fft_inplace(Mloc, scr, lg, ncol >> 1, +1, tws);
                push_pairs(Mloc, Rin, true, -1);
            } else {
                for (int i = wtid; i < ncol << lg; i += ntw) {
                    const int q = i >> lg, n = i & (ns - 1);
                    const int k = (n < (ns >> 1)) ? n : n - ns;
                    Mloc[i] = (k >= -ks && k <= ks) ? uhl[q * nk + k + ks] : mk<R>(0, 0);
                }
                __syncthreads();
                col_fft_inplace(Mloc, scr, lg, ncol, +1, tws);
                push_columns(Mloc, Rin, -1);
            }
        }
        cl.sync();

        int done = 0;
        int st = ST_RUNNING;
        double Jlast = 0.0;
        // The scalars of a step: the sums of the column partials in a fixed order (every rank the
        // same bits), J, L^dag_2, the next T and 2 pi / T, and the freeze decision, taken once so
        // that the other threads compare ints; written to red[0..3] by one lane.  Called by one
        // whole warp.
        auto step_scalars = [&]() {
            double sJ, sL;
            sum_partials(part, part + nkx, nkx, sJ, sL);
            if ((tid & 31) == 0) {
                const double J = sJ * d.L;
                const double L2 = sL * d.L * (wT * wT) * kInv2Pi;  // (L / T^2) 2 pi sum
                const double Tn = T - d.dtau * L2;    // explicit Euler for T (Sec. 4.2)
                int sv = ST_RUNNING;
                if (!(J == J) || J > 1e300 || !(T > 0.0)) sv = ST_DIVERGED;
                else if (J < p.tol * p.tol) sv = ST_CONVERGED;
                else if (p.myprec == 1 && p.switch_tol > 0.0 && J <= p.switch_tol * p.switch_tol) sv = ST_SWITCH;
                red[0] = J;
                red[1] = Tn;
                red[2] = 2.0 * 3.14159265358979323846 / Tn;
                reinterpret_cast<int*>(red + 3)[0] = sv;
            }
        };
        // End of a phase: wait until exchange x has delivered its `bytes` to this rank (ax), or a
        // cluster barrier.  The block barrier first: the pushes read local buffers (the
        // transforms' scratch) that the next phase overwrites.
        auto xsync = [&](int x, unsigned bytes) {
            if (!ax) {
                cl.sync();
                return;
            }
            __syncthreads();
            const unsigned bar = xbar0 + 8u * x;
            if (!xdead) {
                if (tid == 0) xbar_arm(bar, bytes);
                xdead = !xbar_wait(bar, (xpar >> x) & 1u, cp.err);
            }
            xpar ^= 1u << x;
        };
        for (int s = 0; s < nsteps; ++s) {
            // ======== phase A: rows, z = u + i u_x, U, p = u u_x, forward (a1-a4) ========
            for (int t0 = 0; t0 < nrow;) {
                int nr = 2, lgnr = 1;
                while (nr * 2 <= cp.rt && nr * 2 <= nrow - t0) {
                    nr *= 2;
                    ++lgnr;
                }
                const int n0 = row0 + t0;
                cpx<R>* A = scr;
                cpx<R>* Bf = scr + (size_t)nr * nx;
                const int np = nr >> 1;
                cpx<R>* z;
                cpx<R>* Y;
                if constexpr (xi) {
                    // u and u_x of a row pair in one transform (xi_zpair, as the row items)
                    const int lgq = lgnr - 1;
                    for (int i = wtid; i < np * nx; i += ntw) {
                        const int J = i >> lgq, pr = i & (np - 1);
                        cpx<R> y = mk<R>(0, 0);
                        if (J <= kx) {
                            const cpx<R>* src = Rin + (size_t)J * rmax + t0 + 2 * pr;
                            y = xi_zpair(src[0], src[1], s_qv[J]);
                        } else if (J >= nx - kx) {
                            const cpx<R>* src = Rin + (size_t)(nx - J) * rmax + t0 + 2 * pr;
                            y = xi_zpair(conj(src[0]), conj(src[1]), -s_qv[nx - J]);
                        }
                        A[(size_t)pr * nx + J] = y;
                    }
                    __syncthreads();
                    z = fft_pair_warp<R, true>(A, Bf, lgnx, np, +1, tws);
                    Y = (z == A) ? Bf : A;
                    for (int i = wtid; i < np * nx; i += ntw) {
                        const int pr = i >> lgnx, m = i & (nx - 1);
                        R ua, ub, uxa, uxb;
                        xi_zsplit(z[i], z[(size_t)pr * nx + ((nx - m) & (nx - 1))], ua, ub, uxa, uxb);
                        Ul[(size_t)(t0 + 2 * pr) * nx + m] = ua;
                        Ul[(size_t)(t0 + 2 * pr + 1) * nx + m] = ub;
                        Y[i] = mk<R>(ua * uxa, ub * uxb);
                    }
                } else {
                    for (int i = wtid; i < nr * nx; i += ntw) {
                        const int J = i >> lgnr, r = i & (nr - 1);
                        cpx<R> zz = mk<R>(0, 0);
                        if (J <= kx) zz = scale(Rin[(size_t)J * rmax + t0 + r], (R)1 - s_qv[J]);
                        else if (J >= nx - kx) zz = scale(conj(Rin[(size_t)(nx - J) * rmax + t0 + r]), (R)1 + s_qv[nx - J]);
                        A[(size_t)r * nx + J] = zz;
                    }
                    __syncthreads();
                    z = fft_warp<R, true>(A, Bf, lgnx, nr, +1, tws);
                    Y = (z == A) ? Bf : A;
                    for (int i = wtid; i < np * nx; i += ntw) {
                        const int pr = i >> lgnx, m = i & (nx - 1);
                        const cpx<R> za = z[(size_t)(2 * pr) * nx + m];
                        const cpx<R> zb = z[(size_t)(2 * pr + 1) * nx + m];
                        Ul[(size_t)(t0 + 2 * pr) * nx + m] = za.x;
                        Ul[(size_t)(t0 + 2 * pr + 1) * nx + m] = zb.x;
                        Y[i] = mk<R>(za.x * za.y, zb.x * zb.y);
                    }
                }
                __syncthreads();
                cpx<R>* F = fft_pair_warp<R, true>(Y, z, lgnx, np, -1, tws);
                const int lgp = lgnr - 1;
                for (int i = wtid; i < (nkx << lgp); i += ntw) {
                    const int j = i >> lgp, pr = i & (np - 1);
                    if (xi && j == 0) continue;  // the zero column of the subspace
                    const cpx<R> yj = F[(size_t)pr * nx + j];
                    const cpx<R> ym = conj(F[(size_t)pr * nx + ((nx - j) & (nx - 1))]);
                    const cpx<R> sm = yj + ym, df = yj - ym;
                    xput(Mloc + (size_t)own_slot(j) * ns + n0 + 2 * pr, own_rank(j), 0, scale(sm, h),
                         mk<R>(df.y * h, -df.x * h));
                }
                __syncthreads();
                t0 += nr;
            }
            xsync(0, bx_A);

            // ======== phase B: columns, r_hat, partials, rho = s-inverse of i q r_hat ========
            if (ncol > 0 && xi) {
                // centre-symmetric subspace: one s-transform per column pair (col_pair_item)
                const int npair = ncol >> 1;
                for (int i = wtid; i < npair << lg; i += ntw) {
                    const int pp = i >> lg, n = i & (ns - 1);
                    // a ghost second column (past Kx) holds no data: it packs zeros
                    const bool hasb = colj(2 * pp + 1) <= kx;
                    scr[i] = mk<R>(Mloc[((2 * pp) << lg) + n].y, hasb ? Mloc[((2 * pp + 1) << lg) + n].y : (R)0);
                }
                __syncthreads();
                col_fft_inplace(scr, Mloc, lg, npair, -1, tws);
                const R wTr = (R)wT;
                for (int pp = 0; pp < npair; ++pp) {
                    const int ja = colj(2 * pp), jb = ja + 1;
                    const bool hasb = jb <= kx;
                    ColAcc<R> acc[2];
                    if (tid < COL_ACC_LANES) {
                        const R lin_a = s_lin[ja], q_a = s_qv[ja];
                        const R lin_b = hasb ? s_lin[jb] : (R)0, q_b = hasb ? s_qv[jb] : (R)0;
                        const cpx<R>* Cp = scr + (pp << lg);
                        for (int n = tid; n < ns; n += COL_ACC_LANES) {
                            const int k = (n < (ns >> 1)) ? n : n - ns;
                            cpx<R> x = mk<R>(0, 0);
                            if (k >= -ks && k <= ks) {
                                const cpx<R> ck = Cp[n], cm = Cp[(ns - n) & (ns - 1)];
                                const R bk = -(R)k * wTr;
                                const cpx<R> pa = xi_split_a(ck, cm);
                                const cpx<R> ua = uhl[(2 * pp) * nk + k + ks];
                                const cpx<R> ra = mk<R>(lin_a * ua.x - bk * ua.y - pa.x, lin_a * ua.y + bk * ua.x - pa.y);
                                rhl[(2 * pp) * nk + k + ks] = ra;
                                acc[0].add(ua, ra, k);
                                cpx<R> xb = mk<R>(0, 0);
                                if (hasb) {
                                    const cpx<R> pb = xi_split_b(ck, cm);
                                    const cpx<R> ub = uhl[(2 * pp + 1) * nk + k + ks];
                                    const cpx<R> rb = mk<R>(lin_b * ub.x - bk * ub.y - pb.x, lin_b * ub.y + bk * ub.x - pb.y);
                                    rhl[(2 * pp + 1) * nk + k + ks] = rb;
                                    acc[1].add(ub, rb, k);
                                    xb = mk<R>(-q_b * rb.y, q_b * rb.x);
                                }
                                x = xi_join_real(mk<R>(-q_a * ra.y, q_a * ra.x), xb);
                            }
                            Mloc_a[(pp << lg) + n] = mk<RA>((RA)x.x, (RA)x.y);
                        }
                    }
                    block_reduce2(acc[0], acc[1], red);
                    if (tid < C) {
                        xpart(ja, tid, acc[0].part_J(2.0));
                        xpart(nkx + ja, tid, acc[0].part_L(2.0));
                        if (hasb) {
                            xpart(jb, tid, acc[1].part_J(2.0));
                            xpart(nkx + jb, tid, acc[1].part_L(2.0));
                        }
                    }
                }
                __syncthreads();
                // inverse of the pairs of i q r_hat (Mloc holds the spectra, scr is scratch)
                push_pairs(fft_col_warp<RA, true>(Mloc_a, scr_a, lg, npair, +1, tws_a), Rin_a, false, 1);
            } else if (ncol > 0) {
                col_fft_inplace(Mloc, scr, lg, ncol, -1, tws);
                const R wTr = (R)wT;
                // columns in pairs: one block reduction for two columns' partials.  Element n of a
                // column is accumulated by thread n mod COL_ACC_LANES, as in the item kernels, so
                // the partials do not depend on the block size.
                for (int q0 = 0; q0 < ncol; q0 += 2) {
                    const bool two = q0 + 1 < ncol;
                    ColAcc<R> acc[2];
                    if (tid < COL_ACC_LANES) {
                        for (int n = tid; n < ns; n += COL_ACC_LANES) {
                            const int k = (n < (ns >> 1)) ? n : n - ns;
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                if (t == 1 && !two) break;
                                const int q = q0 + t;
                                const int j = rank + q * C;
                                cpx<R> x = mk<R>(0, 0);
                                if (k >= -ks && k <= ks) {
                                    const R a_lin = s_lin[j], rq = s_qv[j];
                                    const cpx<R> ph = Mloc[(q << lg) + n];
                                    const cpx<R> u = uhl[q * nk + k + ks];
                                    const R bk = -(R)k * wTr;
                                    const cpx<R> r = mk<R>(a_lin * u.x - bk * u.y - ph.x, a_lin * u.y + bk * u.x - ph.y);
                                    rhl[q * nk + k + ks] = r;
                                    acc[t].add(u, r, k);
                                    x = mk<R>(-rq * r.y, rq * r.x);
                                }
                                scr_a[(q << lg) + n] = mk<RA>((RA)x.x, (RA)x.y);
                            }
                        }
                    }
                    if (two) block_reduce2(acc[0], acc[1], red);
                    else block_reduce(acc[0], red);
                    if (tid < C) {
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            if (t == 1 && !two) break;
                            const int j = rank + (q0 + t) * C;
                            const double wj = (j == 0) ? 1.0 : 2.0;
                            xpart(j, tid, acc[t].part_J(wj));
                            xpart(nkx + j, tid, acc[t].part_L(wj));
                        }
                    }
                }
                __syncthreads();
                // inverse of i q r_hat (scr holds the spectra, Mloc is scratch), then push rho
                push_columns(fft_col_warp<RA, true>(scr_a, Mloc_a, lg, ncol, +1, tws_a), Rin_a, 1);
            }
            xsync(1, bx_B);

            // ======== phase A': rows, r_x, w = u r_x, forward (a7, a8) ========
            // A float state with an extra warp (sa): the work warps run the phase alone,
            // synchronised by a named barrier, while the extra warp forms this step's scalars;
            // the partials of J and L^dag_2 are complete since the barrier that closed phase B.
            if (sa && tid >= ntw) {
                step_scalars();
            } else
            for (int t0 = 0; t0 < nrow;) {
                int nr = 2, lgp = 0;
                while (nr * 2 <= cp.rt && nr * 2 <= nrow - t0) {
                    nr *= 2;
                    ++lgp;
                }
                const int np = nr >> 1;
                const int n0 = row0 + t0;
                cpx<RA>* A = scr_a;
                cpx<RA>* Bf = scr_a + (size_t)nr * nx;
                for (int i = wtid; i < np * nx; i += ntw) {
                    const int J = i >> lgp, pr = i & (np - 1);
                    cpx<RA> z = mk<RA>(0, 0);
                    if (J <= kx) {
                        const cpx<RA>* src = Rin_a + (size_t)J * rmax + t0 + 2 * pr;
                        z = src[0] + mul_i(src[1], 1);
                    } else if (J >= nx - kx) {
                        const cpx<RA>* src = Rin_a + (size_t)(nx - J) * rmax + t0 + 2 * pr;
                        z = conj(src[0]) + mul_i(conj(src[1]), 1);
                    }
                    A[(size_t)pr * nx + J] = z;
                }
                wsync();
                cpx<RA>* z = fft_pair_warp<RA, true>(A, Bf, lgnx, np, +1, tws_a, wn);
                cpx<RA>* Y = (z == A) ? Bf : A;
                for (int i = wtid; i < np * nx; i += ntw) {
                    const int pr = i >> lgnx, m = i & (nx - 1);
                    const cpx<RA> rx = z[i];
                    Y[i] = mk<RA>((RA)Ul[(size_t)(t0 + 2 * pr) * nx + m] * rx.x,
                                  (RA)Ul[(size_t)(t0 + 2 * pr + 1) * nx + m] * rx.y);
                }
                wsync();
                cpx<RA>* F = fft_pair_warp<RA, true>(Y, z, lgnx, np, -1, tws_a, wn);
                for (int i = wtid; i < (nkx << lgp); i += ntw) {
                    const int j = i >> lgp, pr = i & (np - 1);
                    if (xi && j == 0) continue;
                    const cpx<RA> yj = F[(size_t)pr * nx + j];
                    const cpx<RA> ym = conj(F[(size_t)pr * nx + ((nx - j) & (nx - 1))]);
                    const cpx<RA> sm = yj + ym, df = yj - ym;
                    xput(Mloc2_a + (size_t)own_slot(j) * ns + n0 + 2 * pr, own_rank(j), 2, scale(sm, h_a),
                         mk<RA>(df.y * h_a, -df.x * h_a));
                }
                wsync();
                t0 += nr;
            }
            xsync(2, bx_Aa);

            // ======== phase B': J, L2, freeze test, G_hat, update, v = s-inverse (a9, a10) ===
            // The last warp sums the partials and its first lane forms J, L^dag_2 and the next T,
            // 2 pi / T (step_scalars), while the other warps run the s-transform of w_hat (its
            // result is not used when the loop stops at this step); a float state with an extra
            // warp has them ready from phase A' (sa).  A float transform is warp-owned: the last
            // warp owns none for up to (warps - 1) columns and only joins its closing barrier.  A
            // double transform runs on the other warps alone (nfft threads), synchronised by a
            // named barrier.
            constexpr bool kFloatAdj = sizeof(RA) == 4;
            const int nfft = nt - 32;  // threads of a double transform of w_hat
            if (!sa && tid >= nt - 32) {
                step_scalars();
            } else if constexpr (!kFloatAdj) {
                if (tid < nfft) {
                    if (ncol > 0 && xi) {
                        // pairs: the imaginary columns of W packed two to a transform
                        for (int i = tid; i < (ncol >> 1) << lg; i += nfft) {
                            const int pp = i >> lg, n = i & (ns - 1);
                            const bool hasb = colj(2 * pp + 1) <= kx;
                            scr_a[i] = mk<RA>(Mloc2_a[((2 * pp) << lg) + n].y,
                                              hasb ? Mloc2_a[((2 * pp + 1) << lg) + n].y : (RA)0);
                        }
                        part_sync(nfft);
                        col_fft_inplace(scr_a, Mloc2_a, lg, ncol >> 1, -1, tws_a, nfft);
                    } else if (ncol > 0) {
                        col_fft_inplace(Mloc2_a, scr_a, lg, ncol, -1, tws_a, nfft);
                    }
                }
            }
            if (kFloatAdj && ncol > 0) {
                if (xi) {
                    for (int i = wtid; i < (ncol >> 1) << lg; i += ntw) {
                        const int pp = i >> lg, n = i & (ns - 1);
                        const bool hasb = colj(2 * pp + 1) <= kx;
                        scr_a[i] = mk<RA>(Mloc2_a[((2 * pp) << lg) + n].y,
                                          hasb ? Mloc2_a[((2 * pp + 1) << lg) + n].y : (RA)0);
                    }
                    __syncthreads();
                    col_fft_inplace(scr_a, Mloc2_a, lg, ncol >> 1, -1, tws_a);
                } else {
                    col_fft_inplace(Mloc2_a, scr_a, lg, ncol, -1, tws_a);
                }
            }
            __syncthreads();
            const double J = red[0], Tnext = red[1], wTnext = red[2];
            st = reinterpret_cast<const int*>(red + 3)[0];
            __syncthreads();
            Jlast = J;
            if (st != ST_RUNNING) break;  // uniform: every rank computed the same J and T
            if (ncol > 0 && xi) {
                // pairs (col_pair_item): G_hat of both columns from the packed transform in scr,
                // no projection needed (the split keeps the symmetry exactly); the new u_hat of
                // both packed into Mloc2 for one inverse transform
                const int npair = ncol >> 1;
                const R wTr = (R)wT;
                const R dt = (R)d.dtau;
                const R wT2 = wTr * wTr;
                const RA wTa = (RA)wT;
                for (int i = wtid; i < npair << lg; i += ntw) {
                    const int pp = i >> lg, n = i & (ns - 1);
                    const int k = (n < (ns >> 1)) ? n : n - ns;
                    cpx<R> x = mk<R>(0, 0);
                    if (k >= -ks && k <= ks) {
                        const int ja = colj(2 * pp), jb = ja + 1;
                        const cpx<RA> ck = scr_a[i], cm = scr_a[(pp << lg) + ((ns - n) & (ns - 1))];
                        const RA bk = (RA)k * wTa;
                        const R kk2 = (R)k * (R)k;
                        auto update = [&](int q, int j, cpx<RA> wh) {
                            const RA a_lin = s_lina[j];
                            const cpx<R> rr = rhl[q * nk + k + ks];
                            const cpx<RA> r = mk<RA>((RA)rr.x, (RA)rr.y);
                            const cpx<RA> Ga = mk<RA>(a_lin * r.x - bk * r.y + wh.x, a_lin * r.y + bk * r.x + wh.y);
                            const cpx<R> G = mk<R>((R)Ga.x, (R)Ga.y);
                            R f = dt;
                            if (d.scheme == 1) f = dt / ((R)1 + dt * (kk2 * wT2 + s_cq[j]));
                            cpx<R> u = uhl[q * nk + k + ks];
                            u = u - scale(G, f);
                            uhl[q * nk + k + ks] = u;
                            return u;
                        };
                        const cpx<R> ua = update(2 * pp, ja, xi_split_a(ck, cm));
                        const cpx<R> ub = (jb <= kx) ? update(2 * pp + 1, jb, xi_split_b(ck, cm)) : mk<R>(0, 0);
                        x = xi_join_imag(ua, ub);
                    }
                    Mloc2[i] = x;
                }
                __syncthreads();
                push_pairs(fft_col_warp<R, true>(Mloc2, scr, lg, npair, +1, tws), Rin, true, 3);
            } else if (ncol > 0) {
                const R wTr = (R)wT;
                const R dt = (R)d.dtau;
                const R wT2 = wTr * wTr;
                const RA wTa = (RA)wT;
                // G_hat = (a + i omega/T) r_hat + F[P(u r_x)], in the adjoint precision
                auto g_hat = [&](int i, int q, int k) {
                    const cpx<RA> wh = Mloc2_a[i];
                    const RA a_lin = s_lina[rank + q * C];
                    const cpx<R> rr = rhl[q * nk + k + ks];
                    const cpx<RA> r = mk<RA>((RA)rr.x, (RA)rr.y);
                    const RA bk = (RA)k * wTa;
                    const cpx<RA> G = mk<RA>(a_lin * r.x - bk * r.y + wh.x, a_lin * r.y + bk * r.x + wh.y);
                    return mk<R>((R)G.x, (R)G.y);
                };
                // double state with more than one element per thread: the band by (k, -k) pairs,
                // which share the IMEX factor ((-k)^2 = k^2 exactly), so a thread divides once for
                // both; the out-of-band elements are zeroed apart (64x128 double 28.48 -> 27.78 us
                // per step, the same bits; the float kernels, where a division is cheap, measured
                // slower with the branch compiled in, so they keep one loop)
                bool paired = false;
                if constexpr (sizeof(R) == 8) paired = (ncol << lg) > ntw;
                if (paired) {
                    const int nh = ks + 1;
                    for (int i = wtid; i < ncol * nh; i += ntw) {
                        const int q = i / nh, k = i - q * nh;
                        R f = dt;
                        if (d.scheme == 1) {
                            const R kk2 = (R)k * (R)k;
                            f = dt / ((R)1 + dt * (kk2 * wT2 + s_cq[rank + q * C]));
                        }
                        auto upd = [&](int kk, int n) {
                            const int e = (q << lg) + n;
                            const cpx<R> G = g_hat(e, q, kk);
                            cpx<R> u = uhl[q * nk + kk + ks];
                            u = u - scale(G, f);
                            uhl[q * nk + kk + ks] = u;
                            scr[e] = u;
                        };
                        upd(k, k);
                        if (k > 0) upd(-k, ns - k);
                    }
                    for (int i = wtid; i < ncol << lg; i += ntw) {
                        const int n = i & (ns - 1);
                        const int k = (n < (ns >> 1)) ? n : n - ns;
                        if (k < -ks || k > ks) scr[i] = mk<R>(0, 0);
                    }
                } else {
                    for (int i = wtid; i < ncol << lg; i += ntw) {
                        const int q = i >> lg, n = i & (ns - 1);
                        const int k = (n < (ns >> 1)) ? n : n - ns;
                        cpx<R> x = mk<R>(0, 0);
                        if (k >= -ks && k <= ks) {
                            const int j = rank + q * C;
                            const cpx<R> G = g_hat(i, q, k);
                            R f = dt;
                            if (d.scheme == 1) {
                                const R kk2 = (R)k * (R)k;
                                f = dt / ((R)1 + dt * (kk2 * wT2 + s_cq[j]));
                            }
                            cpx<R> u = uhl[q * nk + k + ks];
                            u = u - scale(G, f);
                            uhl[q * nk + k + ks] = u;
                            x = u;
                        }
                        scr[i] = x;
                    }
                }
                __syncthreads();
                push_columns(fft_col_warp<R, true>(scr, Mloc2, lg, ncol, +1, tws), Rin, 3);
            }
            T = Tnext;
            wT = wTnext;
            ++done;
            xsync(3, bx_Ba);
        }

        // ---- write the loop back: band of the owned columns, mixed values of the own rows
        for (int i = tid; i < ncol * nk; i += nt) {
            const int q = i / nk, kk = i - q * nk;
            const int j = colj(q);
            if (j <= kx) p.uh[bo + (size_t)j * nk + kk] = uhl[i];
        }
        for (int i = tid; i < nkx * nrow; i += nt) {
            const int j = i / nrow, r = i - j * nrow;
            Mg[(size_t)j * ns + row0 + r] = Rin[(size_t)j * rmax + r];
        }
        if (rank == 0 && tid == 0) {
            p.T[(size_t)par0 * B + b] = T;
            p.T[(size_t)(par0 ^ 1) * B + b] = T;
            p.wT[(size_t)par0 * B + b] = wT;
            p.wT[(size_t)(par0 ^ 1) * B + b] = wT;
            p.steps[b] += done;
            if (done > 0 || st != ST_RUNNING) p.sqrtJ[b] = sqrt(Jlast);
            if (st != ST_RUNNING) p.status[b] = st;
        }
        cl.sync();
    }
    cp_async_wait();  // a cluster whose loops were all skipped still has its table copies
}

}  // namespace ks
