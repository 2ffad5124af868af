// ks_items.cuh - per-CTA work items of one tau-step of the KS loop descent.
//
// One tau-step (Sec. 4.2 of the paper; steps listed in order):
//   a1  u_x = i q_j u_hat (spectral derivative)
//   a2  inverse 2-D transform of u_hat and (u_x)_hat to the grid
//   a3  pointwise product u u_x
//   a4  forward 2-D transform of the product, truncated to the 2/3 band
//   a5  r_hat = (-i w_k / T + q_j^2 - q_j^4) u_hat - F[P(u u_x)]               (Eq. KS_R)
//   a6  J = L sum |r_hat|^2 and L^dag_2 = (L/T^2) sum Re(conj(i w_k u_hat) r_hat)
//   a7  r_x = inverse transform of i q_j r_hat
//   a8  forward transform of u r_x, truncated
//   a9  G_hat = (+i w_k / T + q_j^2 - q_j^4) r_hat + F[P(u r_x)] = L^dag_1 r    (Eq. KS_L_dagger)
//   a10 u_hat -= dtau G_hat (explicit) or dtau G_hat / (1 - dtau Lambda_jk(T)) (IMEX, Sec. 4.2),
//       T -= dtau L^dag_2 (explicit Euler)
//
// The 2-D transforms are split into x-passes (one grid row n at a time, length Nx) and
// s-passes (one retained x-mode column j at a time, length Ns).  The band state lives in a
// half spectrum j = 0..Kx, k = -Ks..Ks.  Between the passes the data sits in the "mixed"
// array M[b][j][n] (x-mode j, time sample n).  A step is four phases, each a set of
// independent CTA work items:
//   ROW_NONLIN  (rows)    : M = v (u_hat s-inverted) -> u, u_x rows -> U grid, p = u u_x -> M = P
//   COL_RESID   (columns) : M = P -> r_hat (a5), partial J / L^dag_2 (a6), M = s-inverse of i q r_hat
//   ROW_ADJ     (rows)    : M = rho -> r_x rows, w = u r_x -> M = W
//   COL_UPDATE  (columns) : M = W -> G_hat (a9), update (a10), M = s-inverse of the new u_hat
// plus the analysis (grid -> band) and synthesis (band -> grid) items used at the boundary.
//
// Every loop inside an item is a CTA-strided loop separated by KS_SYNC(), so the source also
// compiles as sequential host code (KS_HOST_EMULATION) for index checks.
#pragma once

#include <cstdint>
#include <cmath>

#ifdef KS_HOST_EMULATION
#define KS_HDX inline
#define KS_HD inline
#define KS_TID 0
#define KS_NT 1
#define KS_SYNC() ((void)0)
#else
#define KS_HDX __host__ __device__ inline  // also called by the host code that sizes launches
#define KS_HD __device__ __forceinline__
#define KS_TID ((int)threadIdx.x)
#define KS_NT ((int)blockDim.x)
#define KS_SYNC() __syncthreads()
#endif

namespace ks {

constexpr int NMAX = 1024;  // largest transform length (Nx and Ns)
constexpr int LGNMAX = 10;

// per-loop status values (match the public header)
constexpr int ST_RUNNING = 0;
constexpr int ST_CONVERGED = 1;
constexpr int ST_STEP_CAP = 2;
constexpr int ST_STALLED = 3;
constexpr int ST_DIVERGED = 4;
constexpr int ST_SWITCH = 5;  // internal: float phase reached the switch criterion

template <typename R>
struct cpx {
    R x, y;
};

template <typename R>
KS_HD cpx<R> mk(R a, R b) {
    cpx<R> c;
    c.x = a;
    c.y = b;
    return c;
}
template <typename R>
KS_HD cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R>
KS_HD cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R>
KS_HD cpx<R> cmul(cpx<R> a, cpx<R> b) {
    return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
KS_HD cpx<R> conj(cpx<R> a) { return mk<R>(a.x, -a.y); }
template <typename R>
KS_HD cpx<R> scale(cpx<R> a, R s) { return mk<R>(a.x * s, a.y * s); }
// multiply by i*sgn (sgn = +1 or -1)
template <typename R>
KS_HD cpx<R> mul_i(cpx<R> a, int sgn) { return sgn > 0 ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x); }

// fused multiply-add a * b + c with one rounding, in either precision
KS_HD double fmx(double a, double b, double c) { return fma(a, b, c); }
KS_HD float fmx(float a, float b, float c) { return fmaf(a, b, c); }

// v0 + w v (complex) as four fused multiply-adds
template <typename R>
KS_HD cpx<R> cfma(cpx<R> v0, cpx<R> w, cpx<R> v) {
    return mk<R>(fmx(w.x, v.x, fmx(-w.y, v.y, v0.x)), fmx(w.x, v.y, fmx(w.y, v.x, v0.y)));
}

// 2 a - b (complex) as two fused multiply-adds
template <typename R>
KS_HD cpx<R> twice_minus(cpx<R> a, cpx<R> b) {
    return mk<R>(fmx((R)2, a.x, -b.x), fmx((R)2, a.y, -b.y));
}

// Radix-4 butterfly of a decimation-in-time pass with twiddles w1, w2, w3 on v1, v2, v3
// (dir: sign of the exponent).  The twiddle products are fused into the additions that follow
// them: t0 = v0 + w2 v2 and t2 = w1 v1 + w3 v3 as fused multiply-adds, t1 = v0 - w2 v2 and
// w1 v1 - w3 v3 as 2 v0 - t0 and 2 w1 v1 - t2: 24 floating-point operations for the butterfly
// where separate products and additions take 28 (the FP64 pipe bounds the double path).
template <typename R>
KS_HD void bfly4_tw(cpx<R> v0, cpx<R> v1, cpx<R> v2, cpx<R> v3, cpx<R> w1, cpx<R> w2, cpx<R> w3,
                    int dir, cpx<R>& o0, cpx<R>& o1, cpx<R>& o2, cpx<R>& o3) {
    const cpx<R> a1 = cmul(v1, w1);
    const cpx<R> t0 = cfma(v0, w2, v2);
    const cpx<R> t1 = twice_minus(v0, t0);
    const cpx<R> t2 = cfma(a1, w3, v3);
    const cpx<R> t3 = mul_i(twice_minus(a1, t2), dir);
    o0 = t0 + t2;
    o1 = t1 + t3;
    o2 = t0 - t2;
    o3 = t1 - t3;
}

// ---- compensated float arithmetic (error-free transformations) -----------------------------
// A float-float value hi + lo (|lo| <= ulp(hi) / 2).  Sums use Knuth's TwoSum, products use an
// FMA to recover the rounding error of a * b exactly.  The float path keeps its reductions of
// J and L^dag_2 in this form, on the FP32 pipe, and widens only the final value to double.
struct ff {
    float hi, lo;
};
KS_HD ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    ff r;
    r.hi = s;
    r.lo = e;
    return r;
}
KS_HD ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    const float e = s.lo + (a.lo + b.lo);
    return two_sum(s.hi, e);
}
KS_HD ff two_prod(float a, float b) {
    const float p = a * b;
    ff r;
    r.hi = p;
    r.lo = fmaf(a, b, -p);
    return r;
}

// Per-column partial of the two reductions: double, or float-float in the float path (8 bytes
// either way, so one buffer serves both precisions).
template <typename R>
struct PartT {
    typedef double type;
};
template <>
struct PartT<float> {
    typedef ff type;
};

// Per-thread accumulation of |r_hat|^2 and k Im(conj(u_hat) r_hat) over the modes of one column.
template <typename R>
struct ColAcc;
template <>
struct ColAcc<double> {
    double J = 0.0, L = 0.0;
    KS_HD void add(cpx<double> u, cpx<double> r, int k) {
        J += r.x * r.x + r.y * r.y;
        L += (double)k * (u.x * r.y - u.y * r.x);
    }
    KS_HD double part_J(double wj) const { return wj * J; }
    KS_HD double part_L(double wj) const { return wj * L; }
};
template <>
struct ColAcc<float> {
    ff J = {0.f, 0.f}, L = {0.f, 0.f};
    KS_HD void add(cpx<float> u, cpx<float> r, int k) {
        J = ff_add(J, ff_add(two_prod(r.x, r.x), two_prod(r.y, r.y)));
        ff q = two_prod(u.y, r.x);
        q.hi = -q.hi;
        q.lo = -q.lo;
        const ff d = ff_add(two_prod(u.x, r.y), q);
        const float kf = (float)k;  // exact: |k| < 2^24
        ff t = two_prod(kf, d.hi);
        t.lo = fmaf(kf, d.lo, t.lo);
        L = ff_add(L, t);
    }
    KS_HD ff part_J(double wj) const { return wj == 1.0 ? J : ff{2.f * J.hi, 2.f * J.lo}; }
    KS_HD ff part_L(double wj) const { return wj == 1.0 ? L : ff{2.f * L.hi, 2.f * L.lo}; }
};

KS_HD double widen(double v) { return v; }
KS_HD double widen(ff v) { return (double)v.hi + (double)v.lo; }

struct RowItem {
    int b, n0, nr, lgnr;  // loop, first row, rows in the tile (even power of two), log2 nr
};

// Shape of the batch (shared by all loops of a handle).
struct Dims {
    int B;         // loops
    int nx, lgnx;  // Nx = 2^lgnx
    int kx, nkx;   // Kx = Nx / 3, nkx = Kx + 1 retained x-modes (half spectrum)
    double L;
    double dtau;
    int scheme;    // 0 explicit, 1 IMEX
    double hx;     // 0.5 / Nx (forward x-pass scale with the pair split)
};

// Device buffers of one precision, plus the per-loop scalars (always double / int).
template <typename R>
struct Bufs {
    const int* ns;          // [B] Ns_b
    const int* lgns;        // [B] log2 Ns_b
    const int* ks;          // [B] Ks_b = Ns_b / 3
    const long long* boff;  // [B] band offset (complex elements); band is [j][kk], kk = k + Ks
    const long long* moff;  // [B] mixed-array offset (complex elements); [j][n]
    const long long* goff;  // [B] grid offset (real elements); [n][m]
    cpx<R>* uh;             // band state u_hat
    cpx<R>* rh;             // band residual r_hat
    cpx<R>* gh;             // band adjoint G_hat (gradient calls only)
    cpx<R>* M;              // mixed array
    R* U;                   // grid u (kept from ROW_NONLIN for ROW_ADJ)
    R* io;                  // grid in/out for analysis / synthesis items
    double* T;              // [2][B] period, double-buffered by step parity
    double* wT;             // [2][B] 2 pi / T, same parity as T
    typename PartT<R>::type* Jpart;   // [B][nkx] per-column partial of sum w_j |r_hat|^2
    typename PartT<R>::type* L2part;  // [B][nkx] per-column partial of sum w_j k Im(conj(u_hat) r_hat)
    int* status;            // [B]
    const int* prec;        // [B] 0 double, 1 float: the precision the loop currently runs in
    long long* steps;       // [B]
    double* sqrtJ;          // [B]
    const cpx<R>* tw;       // [NMAX] exp(+2 pi i t / NMAX)
    const R* qv;            // [nkx] q_j = 2 pi j / L in this precision
    const R* lin;           // [nkx] q_j^2 - q_j^4 (symbol of -u_xx - u_xxxx)
    const R* cq;            // [nkx] q_j^4 (q_j^2 - 1)^2 (x part of -Lambda_jk)
    const R* insv;          // [B] 1 / Ns_b
    const RowItem* rows;    // row work items
    const int* colorder;    // loop order of the column items (longest Ns first)
    int myprec;             // precision of this kernel set
    int par;                // step parity: T read from T[par], written to T[par ^ 1]
    double tol;             // freeze a loop once sqrt(J) < tol
    double switch_tol;      // float phase of a mixed descent: freeze as ST_SWITCH once sqrt(J) <= switch_tol
    int check_active;       // 1: skip loops that are not running in this precision
    int xi;                 // 1: descent restricted to the Xi-invariant (centre-symmetric) subspace
    int twsh;               // tw is a compact swizzled shared-memory table: entry t at
                            // tw_swz(t >> twsh) (see load_twiddles_compact); 0 otherwise
    int own_frozen_only;    // cluster kernel: 1 = carry T forward only for frozen loops of this
                            // precision (the other precision's launch runs concurrently and
                            // carries its own)
    int step_scalars;       // 1 (tau-steps): the ROW_ADJ launch forms each running loop's step
                            // scalars (loop_scalars, loops_scalars) for the COL_UPDATE items
                            // that follow
};

// Projection onto the loops invariant under Xi: (x, s) -> (-x, s), u -> -u (Sec. 4.1, the
// symmetry of Eq. KS_G).  An invariant loop has u_hat_{j,-k} = -conj(u_hat_{j,k}) in the
// half spectrum, and a zero j = 0 column.  With a the value at (j, k) and m the value at
// (j, -k), the projected value at (j, k) is (a - conj(m)) / 2.  Evaluated at (j, -k) with the
// two arguments exchanged, the result is exactly -conj of it (IEEE subtraction is antisymmetric
// and addition commutative), so a projected band satisfies the relation bit for bit.
template <typename R>
KS_HD cpx<R> xi_pair(cpx<R> a, cpx<R> m) {
    return mk<R>((R)0.5 * (a.x - m.x), (R)0.5 * (a.y + m.y));
}

// ------------------------------------------------------------------------------------
// Batched Stockham FFT in shared memory.
// `cnt` transforms of length n = 2^lg, stored contiguously (stride n) in `a`; `b` is scratch
// of the same size.  dir = -1: X_k = sum_m x_m e^{-2 pi i m k / n}; dir = +1: e^{+...}.
// No scaling.  Radix-4 passes (one radix-2 pass first when lg is odd); natural order in and
// out.  Returns the buffer holding the result (a or b).  The caller synchronises before the
// call; the function synchronises after every pass.
// ------------------------------------------------------------------------------------
// Position of twiddle t in a bank-swizzled shared-memory copy of the table.  A pass of span s
// reads entries t = jm (NMAX / 4s), jm = 0 .. s-1: a large power-of-two stride that puts the
// lanes of a wavefront (8 double or 16 float complex values = 128 bytes) in one bank group.  The
// low bits of the position are XORed with every higher group of as many bits, which spreads any
// such stride over the banks (a permutation of 0 .. NMAX-1; modelled: mean conflict degree of
// these loads 5.1 -> 1.4 for double, 6.6 -> 1.4 for float).
template <typename R>
KS_HD int tw_swz(int t) {
    constexpr int lgE = sizeof(cpx<R>) == 16 ? 3 : 4;  // complex values per 128 bytes, log2
    constexpr int E = 1 << lgE;
    int x = 0;
#pragma unroll
    for (int k = lgE; k < LGNMAX; k += lgE) x ^= t >> k;  // t < NMAX = 2^LGNMAX
    return t ^ (x & (E - 1));
}

template <typename R, bool SWZ = false>
KS_HD cpx<R> twid(const cpx<R>* tw, int t, int dir, int sh = 0) {
    cpx<R> w = tw[SWZ ? tw_swz<R>(t >> sh) : t];
    if (dir < 0) w.y = -w.y;
    return w;
}

// Row skew of a transform buffer.  The element loops around the x-transforms address their
// buffers row by row with the rows fastest (the gathers of the mixed values, the splits of the
// spectra), so consecutive lanes touch one element of each row at a stride of Nx elements: all on
// one bank.  Element x of transform (row) f therefore sits at f n + (x ^ row_skew(f, n)), the
// column index XORed with the row's low bits (below the 128 bytes of E elements, and below n), so
// the lanes of such a loop spread over E banks.  Only the buffers that those loops fill (the
// input of an inverse x-transform) or read (the output of a forward one) are skewed: the
// transform reads its input (SKI) or writes its output (SKO) through the same map, one XOR in its
// first or last pass.  Addresses only: the arithmetic, hence every result, is unchanged.
// Float buffers only: on GB300 the per-phase float steps ran about 3% faster with it, while the
// double ones (8 elements per 128 bytes, pipe-bound FP64 transforms) did not gain, so for double
// the skew is 0 and the XORs fold away.
template <typename R>
KS_HD int row_skew(int f, int n) {
    if constexpr (sizeof(R) != 4) return 0;
    constexpr int E = 128 / (int)sizeof(cpx<R>);
    return f & ((n < E ? n : E) - 1);
}

// Barrier of the first nthr threads of the block (a multiple of 32): a plain block barrier when
// that is the whole block, else named barrier 1, which the other warps never use.
KS_HD void part_sync(int nthr) {
#ifdef KS_HOST_EMULATION
    (void)nthr;
#else
    if (nthr == (int)blockDim.x) __syncthreads();
    else asm volatile("bar.sync 1, %0;\n" ::"r"(nthr) : "memory");
#endif
}

// SWZ: the table is the swizzled shared-memory copy (see tw_swz); the global table is not.
// nthr > 0: only the first nthr threads (a multiple of 32) run the transform and meet at
// part_sync(nthr); every one of them must call it.  The arithmetic is the same either way.
// twsh: the swizzled table is compact (entry t at tw_swz(t >> twsh)).
// SKI / SKO: the input / output is row-skewed (row_skew).
template <typename R, bool SWZ = false, bool SKI = false, bool SKO = false>
KS_HD cpx<R>* fft_batch(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir, const cpx<R>* tw,
                        int nthr = 0, int twsh = 0) {
#ifdef KS_HOST_EMULATION
    const int NT = KS_NT;
#else
    const int NT = nthr > 0 ? nthr : KS_NT;
#endif
    const int n = 1 << lg;
    int span = 1;  // size of the sub-transforms completed so far
    int p = lg;
    bool first = true;
    if (p & 1) {
        // radix-2 pass with span 1: no twiddles (never the last pass: n >= 8)
        const int nb = n >> 1;
        const int total = cnt * nb;
        for (int i = KS_TID; i < total; i += NT) {
            const int f = i >> (lg - 1);
            const int j = i & (nb - 1);
            const int si = SKI ? row_skew<R>(f, n) : 0;
            const cpx<R>* s = a + (size_t)f * n;
            cpx<R>* d = b + (size_t)f * n;
            const cpx<R> v0 = s[j ^ si], v1 = s[(j + nb) ^ si];
            d[2 * j] = v0 + v1;
            d[2 * j + 1] = v0 - v1;
        }
        if (nthr > 0) part_sync(nthr);
        else KS_SYNC();
        cpx<R>* t = a;
        a = b;
        b = t;
        span = 2;
        p -= 1;
        first = false;
    }
    while (p > 0) {
        const int nb = n >> 2;
        const int total = cnt * nb;
        const int tu = NMAX / (span * 4);
        const bool ski = SKI && first, sko = SKO && p == 2;
        for (int i = KS_TID; i < total; i += NT) {
            const int f = i >> (lg - 2);
            const int j = i & (nb - 1);
            const int si = ski ? row_skew<R>(f, n) : 0;
            const int so = sko ? row_skew<R>(f, n) : 0;
            const cpx<R>* s = a + (size_t)f * n;
            cpx<R>* d = b + (size_t)f * n;
            const cpx<R> v0 = s[j ^ si], v1 = s[(j + nb) ^ si], v2 = s[(j + 2 * nb) ^ si], v3 = s[(j + 3 * nb) ^ si];
            const int jm = j & (span - 1);
            const int od = ((j - jm) << 2) + jm;
            if (span > 1) {
                const int t = jm * tu;
                bfly4_tw(v0, v1, v2, v3, twid<R, SWZ>(tw, t, dir, twsh),
                         twid<R, SWZ>(tw, 2 * t, dir, twsh), twid<R, SWZ>(tw, 3 * t, dir, twsh),
                         dir, d[od ^ so], d[(od + span) ^ so], d[(od + 2 * span) ^ so],
                         d[(od + 3 * span) ^ so]);
            } else {
                const cpx<R> t0 = v0 + v2, t1 = v0 - v2, t2 = v1 + v3;
                const cpx<R> t3 = mul_i(v1 - v3, dir);
                d[od ^ so] = t0 + t2;
                d[(od + 1) ^ so] = t1 + t3;
                d[(od + 2) ^ so] = t0 - t2;
                d[(od + 3) ^ so] = t1 - t3;
            }
        }
        if (nthr > 0) part_sync(nthr);
        else KS_SYNC();
        cpx<R>* t = a;
        a = b;
        b = t;
        span <<= 2;
        p -= 2;
        first = false;
    }
    return a;
}

// Radix-2 variant of fft_batch (every pass a radix-2 pass, natural order in and out, same
// conventions).  A pass has twice the butterflies of a radix-4 pass, so a double transform of
// a single column keeps twice as many warps busy; with the twiddle product fused into the
// additions (v0 + w v1 as four fused multiply-adds, v0 - w v1 as 2 v0 minus that) it costs 3
// floating-point operations per point per radix-2 stage, as the fused radix-4 butterfly does.
template <typename R, bool SWZ = false, bool SKI = false, bool SKO = false>
KS_HD cpx<R>* fft_batch_r2(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir, const cpx<R>* tw,
                           int nthr = 0, int twsh = 0) {
#ifdef KS_HOST_EMULATION
    const int NT = KS_NT;
#else
    const int NT = nthr > 0 ? nthr : KS_NT;
#endif
    const int n = 1 << lg;
    const int nb = n >> 1;
    const int total = cnt * nb;
    for (int span = 1; span < n; span <<= 1) {
        const int tu = NMAX / (span * 2);
        const bool ski = SKI && span == 1, sko = SKO && 2 * span == n;
        for (int i = KS_TID; i < total; i += NT) {
            const int f = i >> (lg - 1);
            const int j = i & (nb - 1);
            const int si = ski ? row_skew<R>(f, n) : 0;
            const int so = sko ? row_skew<R>(f, n) : 0;
            const cpx<R>* s = a + (size_t)f * n;
            cpx<R>* d = b + (size_t)f * n;
            const cpx<R> v0 = s[j ^ si], v1 = s[(j + nb) ^ si];
            const int jm = j & (span - 1);
            const int od = ((j - jm) << 1) + jm;
            if (span > 1) {
                const cpx<R> t = cfma(v0, twid<R, SWZ>(tw, jm * tu, dir, twsh), v1);
                d[od ^ so] = t;
                d[(od + span) ^ so] = twice_minus(v0, t);
            } else {
                d[od ^ so] = v0 + v1;
                d[(od + 1) ^ so] = v0 - v1;
            }
        }
        if (nthr > 0) part_sync(nthr);
        else KS_SYNC();
        cpx<R>* t = a;
        a = b;
        b = t;
    }
    return a;
}

// The s-transforms (columns of the mixed array): in double, radix-2 passes (see fft_batch_r2)
// unless the library is built with KS_COL_RADIX2=0; in float the radix-4 passes of fft_batch.
// Every launch form calls this for its s-transforms, so they keep computing the same bits.
#ifndef KS_COL_RADIX2
#define KS_COL_RADIX2 1
#endif
template <typename R, bool SWZ = false>
KS_HD cpx<R>* fft_col(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir, const cpx<R>* tw,
                      int nthr = 0, int twsh = 0) {
    if constexpr (sizeof(R) == 8 && KS_COL_RADIX2) return fft_batch_r2<R, SWZ>(a, b, lg, cnt, dir, tw, nthr, twsh);
    else return fft_batch<R, SWZ>(a, b, lg, cnt, dir, tw, nthr, twsh);
}

// The x-transforms of row pairs (two real rows packed as one complex row: the forward
// transforms of the products and of the analysis, the inverse ones of r_x and of the synthesis)
// have half as many transforms as the batch has rows; in double they take radix-2 passes
// unless the library is built with KS_PAIR_RADIX2=0.  The transform of z = u + i u_x, one per
// row, keeps the radix-4 passes.  The choice depends on the transform's role only, so every
// launch form computes the same bits.
#ifndef KS_PAIR_RADIX2
#define KS_PAIR_RADIX2 1
#endif
template <typename R, bool SWZ = false, bool SKI = false, bool SKO = false>
KS_HD cpx<R>* fft_pair(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir, const cpx<R>* tw,
                       int nthr = 0, int twsh = 0) {
    if constexpr (sizeof(R) == 8 && KS_PAIR_RADIX2)
        return fft_batch_r2<R, SWZ, SKI, SKO>(a, b, lg, cnt, dir, tw, nthr, twsh);
    else return fft_batch<R, SWZ, SKI, SKO>(a, b, lg, cnt, dir, tw, nthr, twsh);
}

// ------------------------------------------------------------------------------------
// Warp-owned variant of fft_batch: transform f belongs to warp f % warps, which runs every
// pass of it alone and synchronises with __syncwarp() between passes; one block barrier at
// the end.  Same arithmetic in the same order as fft_batch (bit-identical results), far fewer
// block-wide barriers.  Device code only.
//
// Double: an FP64 warp instruction costs the same issue time with idle lanes, and a 64-point
// radix-4 pass has only 16 butterflies per transform, so the double transform runs as
// fft_batch itself (butterflies of all transforms spread over full warps).  A float transform
// is latency-bound and keeps one transform per warp.  (Unrolling the float passes for fixed
// lengths saved little inside the step and cost instruction-cache misses after a launch.)
// ------------------------------------------------------------------------------------
#ifndef KS_HOST_EMULATION
// nthr > 0: only the first nthr threads (a multiple of 32) own transforms and call this; the
// closing barrier is then part_sync(nthr).
template <typename R, bool SWZ = false, bool SKI = false, bool SKO = false>
__device__ __forceinline__ cpx<R>* fft_warp_any(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir,
                                                const cpx<R>* tw, int nthr = 0) {
    const int n = 1 << lg;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (nthr > 0 ? nthr : (int)blockDim.x) >> 5;
    int span = 1;
    int p = lg;
    // this warp's transforms f = w, w + nw, ...; lanes walk (transform, butterfly) jointly
    const int nf = (cnt > w) ? (cnt - w + nw - 1) / nw : 0;
    bool first = true;
    if (p & 1) {
        const int nb = n >> 1;
        for (int i = lane; i < nf * nb; i += 32) {
            const int f = w + (i >> (lg - 1)) * nw, j = i & (nb - 1);
            const int si = SKI ? row_skew<R>(f, n) : 0;
            const cpx<R>* s = a + (size_t)f * n;
            cpx<R>* d = b + (size_t)f * n;
            const cpx<R> v0 = s[j ^ si], v1 = s[(j + nb) ^ si];
            d[2 * j] = v0 + v1;
            d[2 * j + 1] = v0 - v1;
        }
        __syncwarp();
        cpx<R>* t = a;
        a = b;
        b = t;
        span = 2;
        p -= 1;
        first = false;
    }
    while (p > 0) {
        const int nb = n >> 2;
        const int tu = NMAX / (span * 4);
        const bool ski = SKI && first, sko = SKO && p == 2;
        for (int i = lane; i < nf * nb; i += 32) {
            const int f = w + (i >> (lg - 2)) * nw, j = i & (nb - 1);
            const int si = ski ? row_skew<R>(f, n) : 0;
            const int so = sko ? row_skew<R>(f, n) : 0;
            const cpx<R>* s = a + (size_t)f * n;
            cpx<R>* d = b + (size_t)f * n;
            const cpx<R> v0 = s[j ^ si], v1 = s[(j + nb) ^ si], v2 = s[(j + 2 * nb) ^ si], v3 = s[(j + 3 * nb) ^ si];
            const int jm = j & (span - 1);
            const int od = ((j - jm) << 2) + jm;
            if (span > 1) {
                const int t = jm * tu;
                bfly4_tw(v0, v1, v2, v3, twid<R, SWZ>(tw, t, dir), twid<R, SWZ>(tw, 2 * t, dir),
                         twid<R, SWZ>(tw, 3 * t, dir), dir, d[od ^ so], d[(od + span) ^ so],
                         d[(od + 2 * span) ^ so], d[(od + 3 * span) ^ so]);
            } else {
                const cpx<R> t0 = v0 + v2, t1 = v0 - v2, t2 = v1 + v3;
                const cpx<R> t3 = mul_i(v1 - v3, dir);
                d[od ^ so] = t0 + t2;
                d[(od + 1) ^ so] = t1 + t3;
                d[(od + 2) ^ so] = t0 - t2;
                d[(od + 3) ^ so] = t1 - t3;
            }
        }
        __syncwarp();
        cpx<R>* t = a;
        a = b;
        b = t;
        span <<= 2;
        p -= 2;
        first = false;
    }
    if (nthr > 0) part_sync(nthr);
    else __syncthreads();
    return a;
}

// Asynchronous global -> shared copy of N bytes (N = 4, 8 or 16; both addresses N-aligned).
// The issuing thread does not wait for the data, so copies issued back to back share one round
// trip to memory; cp_async_wait() waits for all of the thread's copies (a block barrier after
// it makes them visible to the block).
template <int N>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc) {
    static_assert(N == 4 || N == 8 || N == 16, "cp.async copies 4, 8 or 16 bytes");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gsrc), "n"(N) : "memory");
}

__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The twiddles a transform of length n <= nm reads: entries t of exp(2 pi i t / NMAX) with t a
// multiple of NMAX / n (every pass indexes the table by multiples of NMAX / (4 span) or more, and
// 4 span <= n), hence of NMAX / nm.  Only those entries are copied into the shared-memory copy
// of the table (asynchronously, see cp_async), at their bank-swizzled positions (tw_swz; every
// transform of the cluster and persistent kernels reads the table through it): the values the
// transforms read are unchanged, and the bytes fetched drop by NMAX / nm (8x for 128-point
// columns).
template <typename X>
__device__ __forceinline__ void load_twiddles(cpx<X>* dst, const cpx<X>* src, int nm) {
    const int st = NMAX / nm;
    for (int i = threadIdx.x; i < nm; i += blockDim.x)
        cp_async<sizeof(cpx<X>)>(dst + tw_swz<X>(i * st), src + (size_t)i * st);
}

// The same entries in a compact table of nm slots: entry t = i NMAX / nm at slot tw_swz(i).  The
// transforms read it with twsh = log2(NMAX / nm).  The strides a pass reads are again powers of
// two, which the swizzle spreads over the banks as before.
template <typename X>
__device__ __forceinline__ void load_twiddles_compact(cpx<X>* dst, const cpx<X>* src, int nm) {
    const int st = NMAX / nm;
    for (int i = threadIdx.x; i < nm; i += blockDim.x)
        cp_async<sizeof(cpx<X>)>(dst + tw_swz<X>(i), src + (size_t)i * st);
}

template <typename R, bool SWZ = false, bool SKI = false, bool SKO = false>
__device__ __forceinline__ cpx<R>* fft_warp(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir,
                                            const cpx<R>* tw, int nthr = 0) {
    if constexpr (sizeof(R) == 8) return fft_batch<R, SWZ, SKI, SKO>(a, b, lg, cnt, dir, tw, nthr);
    else return fft_warp_any<R, SWZ, SKI, SKO>(a, b, lg, cnt, dir, tw, nthr);
}

// row-pair x-transforms of the cluster kernel: the double ones as fft_pair (block-wide), the float
// ones warp-owned (the same arithmetic as fft_pair's radix-4 passes)
template <typename R, bool SWZ = false, bool SKI = false, bool SKO = false>
__device__ __forceinline__ cpx<R>* fft_pair_warp(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir,
                                                 const cpx<R>* tw, int nthr = 0) {
    if constexpr (sizeof(R) == 8) return fft_pair<R, SWZ, SKI, SKO>(a, b, lg, cnt, dir, tw, nthr);
    else return fft_warp_any<R, SWZ, SKI, SKO>(a, b, lg, cnt, dir, tw, nthr);
}

// s-transforms of the cluster kernel: the double ones as fft_col (block-wide), the float ones
// warp-owned (the same arithmetic as fft_col's radix-4 passes)
template <typename R, bool SWZ = false>
__device__ __forceinline__ cpx<R>* fft_col_warp(cpx<R>* a, cpx<R>* b, int lg, int cnt, int dir,
                                                const cpx<R>* tw, int nthr = 0) {
    if constexpr (sizeof(R) == 8) return fft_col<R, SWZ>(a, b, lg, cnt, dir, tw, nthr);
    else return fft_warp_any<R, SWZ>(a, b, lg, cnt, dir, tw, nthr);
}
#endif

// First xor distance of the reduction over the per-warp sums held by lanes 0..nw-1 of warp 0
// (the other lanes hold zeros).  At a distance >= nw a lane below nw only meets lanes whose
// values came from lanes >= nw, all zero, so starting below nw gives those lanes the same bits
// in fewer shuffle rounds.
KS_HD int warp0_start(int nw) {
    int o = 16;
    while (o > 1 && o >= nw) o >>= 1;
    return o;
}

#ifndef KS_HOST_EMULATION
// Xor-tree sums of NV values per lane (NV = 2 or 4) over the lanes below 2 o0, starting at xor
// distance o0.  The first levels scatter: at each of the first log2(NV) levels a lane sends half
// of the values it holds and keeps the other half, so a lane adds NV/2, NV/4, ..., 1 values per
// level instead of NV (an FP64 add costs a whole warp-issue slot on this part whatever the lane
// count).  Each value still meets the same xor tree as in a plain butterfly (own + partner at
// every level), and IEEE addition commutes, so every sum has the bits the plain butterfly gives
// at lane 0.  On return the sum of value t sits in lane xor_sum_lane(t, o0) (and its group).
template <int NV>
__device__ __forceinline__ double xor_sum_scatter(const double (&v)[NV], int o0) {
    static_assert(NV == 2 || NV == 4, "two or four values");
    const int l = threadIdx.x & 31;
    double k0, k1;
    int o = o0;
    if constexpr (NV == 4) {
        // level o0: keep (v0, v1) or (v2, v3)
        const bool hi = (l & o) != 0;
        k0 = hi ? v[2] : v[0];
        k1 = hi ? v[3] : v[1];
        const double s0 = __shfl_xor_sync(0xffffffffu, hi ? v[0] : v[2], o);
        const double s1 = __shfl_xor_sync(0xffffffffu, hi ? v[1] : v[3], o);
        k0 += s0;
        k1 += s1;
        o >>= 1;
    } else {
        k0 = v[0];
        k1 = v[1];
    }
    // next level: keep the first or the second of the pair
    const bool hi = (l & o) != 0;
    double k = hi ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, hi ? k0 : k1, o);
    for (o >>= 1; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    return k;
}

// lane holding the sum of value t after xor_sum_scatter<NV>(., o0)
template <int NV>
__device__ __forceinline__ int xor_sum_lane(int t, int o0) {
    return NV == 4 ? (t >> 1) * o0 + (t & 1) * (o0 >> 1) : t * o0;
}
#endif

// Block-wide sum of two doubles per thread (warp shuffles, then one warp over the warp sums);
// red has room for 2 * (warps + 1) doubles.  The result is valid in every thread after the call.
KS_HD void block_sum2(double* red, double& s0, double& s1) {
#ifdef KS_HOST_EMULATION
    (void)red;
#else
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    {
        const double v[2] = {s0, s1};
        const double k = xor_sum_scatter<2>(v, 16);
        if (l == xor_sum_lane<2>(0, 16)) red[2 * w] = k;
        if (l == xor_sum_lane<2>(1, 16)) red[2 * w + 1] = k;
    }
    __syncthreads();
    if (w == 0) {
        const double v[2] = {(l < nw) ? red[2 * l] : 0.0, (l < nw) ? red[2 * l + 1] : 0.0};
        const int o0 = warp0_start(nw);
        if (o0 >= 1) {
            const double k = xor_sum_scatter<2>(v, o0);
            if (l == xor_sum_lane<2>(0, o0)) red[2 * nw] = k;
            if (l == xor_sum_lane<2>(1, o0)) red[2 * nw + 1] = k;
        }
    }
    __syncthreads();
    s0 = red[2 * nw];
    s1 = red[2 * nw + 1];
    __syncthreads();
#endif
}

// Sum of n doubles a[0..n) and c[0..n) in a fixed order, identical in every CTA: lane l adds
// a[l], a[l+32], ... then a shuffle tree.  Every thread of the calling warp gets the sums.
KS_HD void warp_sum_partials(const double* a, const double* c, int n, double& sa, double& sc) {
#ifdef KS_HOST_EMULATION
    sa = 0.0;
    sc = 0.0;
    double la[32] = {0}, lc[32] = {0};
    for (int l = 0; l < 32; ++l)
        for (int i = l; i < n; i += 32) {
            la[l] += a[i];
            lc[l] += c[i];
        }
    for (int o = 16; o > 0; o >>= 1)
        for (int l = 0; l < 32; ++l)
            if ((l & o) == 0 && (l ^ o) < 32) {
                la[l] += la[l ^ o];
                lc[l] += lc[l ^ o];
            }
    sa = la[0];
    sc = lc[0];
#else
    const int l = threadIdx.x & 31;
    double x = 0.0, y = 0.0;
    for (int i = l; i < n; i += 32) {
        x += a[i];
        y += c[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    sa = x;
    sc = y;
#endif
}

// Block-wide reduction of the per-thread column sums (result valid in every thread).
KS_HD void block_reduce(ColAcc<double>& a, double* red) { block_sum2(red, a.J, a.L); }

KS_HD void block_reduce(ColAcc<float>& a, double* redd) {
#ifdef KS_HOST_EMULATION
    (void)a;
    (void)redd;
#else
    float* red = reinterpret_cast<float*>(redd);
    for (int o = 16; o > 0; o >>= 1) {
        ff bJ, bL;
        bJ.hi = __shfl_xor_sync(0xffffffffu, a.J.hi, o);
        bJ.lo = __shfl_xor_sync(0xffffffffu, a.J.lo, o);
        bL.hi = __shfl_xor_sync(0xffffffffu, a.L.hi, o);
        bL.lo = __shfl_xor_sync(0xffffffffu, a.L.lo, o);
        a.J = ff_add(a.J, bJ);
        a.L = ff_add(a.L, bL);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) {
        red[4 * w] = a.J.hi;
        red[4 * w + 1] = a.J.lo;
        red[4 * w + 2] = a.L.hi;
        red[4 * w + 3] = a.L.lo;
    }
    __syncthreads();
    if (w == 0) {
        ff J = {0.f, 0.f}, L = {0.f, 0.f};
        if (l < nw) {
            J.hi = red[4 * l];
            J.lo = red[4 * l + 1];
            L.hi = red[4 * l + 2];
            L.lo = red[4 * l + 3];
        }
        for (int o = warp0_start(nw); o > 0; o >>= 1) {
            ff bJ, bL;
            bJ.hi = __shfl_xor_sync(0xffffffffu, J.hi, o);
            bJ.lo = __shfl_xor_sync(0xffffffffu, J.lo, o);
            bL.hi = __shfl_xor_sync(0xffffffffu, L.hi, o);
            bL.lo = __shfl_xor_sync(0xffffffffu, L.lo, o);
            J = ff_add(J, bJ);
            L = ff_add(L, bL);
        }
        if (l == 0) {
            red[4 * nw] = J.hi;
            red[4 * nw + 1] = J.lo;
            red[4 * nw + 2] = L.hi;
            red[4 * nw + 3] = L.lo;
        }
    }
    __syncthreads();
    a.J.hi = red[4 * nw];
    a.J.lo = red[4 * nw + 1];
    a.L.hi = red[4 * nw + 2];
    a.L.lo = red[4 * nw + 3];
    __syncthreads();
#endif
}

// Two columns' accumulators reduced together: the same shuffle tree and warp-sum order as
// block_reduce for each of them (bit-identical partials), one set of block barriers for both.
// red has room for 4 * (warps + 1) doubles.
KS_HD void block_reduce2(ColAcc<double>& a, ColAcc<double>& b, double* red) {
#ifdef KS_HOST_EMULATION
    block_reduce(a, red);
    block_reduce(b, red);
#else
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    {
        const double v[4] = {a.J, a.L, b.J, b.L};
        const double k = xor_sum_scatter<4>(v, 16);
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (l == xor_sum_lane<4>(t, 16)) red[4 * w + t] = k;
    }
    __syncthreads();
    if (w == 0) {
        double v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = (l < nw) ? red[4 * l + t] : 0.0;
        const int o0 = warp0_start(nw);
        if (o0 >= 2) {
            const double k = xor_sum_scatter<4>(v, o0);
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (l == xor_sum_lane<4>(t, o0)) red[4 * nw + t] = k;
        } else {  // one or two warps: the plain butterfly
            for (int o = o0; o > 0; o >>= 1)
#pragma unroll
                for (int t = 0; t < 4; ++t) v[t] += __shfl_xor_sync(0xffffffffu, v[t], o);
            if (l == 0)
#pragma unroll
                for (int t = 0; t < 4; ++t) red[4 * nw + t] = v[t];
        }
    }
    __syncthreads();
    a.J = red[4 * nw];
    a.L = red[4 * nw + 1];
    b.J = red[4 * nw + 2];
    b.L = red[4 * nw + 3];
    __syncthreads();
#endif
}

KS_HD void block_reduce2(ColAcc<float>& a, ColAcc<float>& b, double* redd) {
#ifdef KS_HOST_EMULATION
    (void)a;
    (void)b;
    (void)redd;
#else
    float* red = reinterpret_cast<float*>(redd);
    ff v[4] = {a.J, a.L, b.J, b.L};
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            ff y;
            y.hi = __shfl_xor_sync(0xffffffffu, v[t].hi, o);
            y.lo = __shfl_xor_sync(0xffffffffu, v[t].lo, o);
            v[t] = ff_add(v[t], y);
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            red[8 * w + 2 * t] = v[t].hi;
            red[8 * w + 2 * t + 1] = v[t].lo;
        }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            v[t].hi = (l < nw) ? red[8 * l + 2 * t] : 0.f;
            v[t].lo = (l < nw) ? red[8 * l + 2 * t + 1] : 0.f;
        }
        for (int o = warp0_start(nw); o > 0; o >>= 1) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                ff y;
                y.hi = __shfl_xor_sync(0xffffffffu, v[t].hi, o);
                y.lo = __shfl_xor_sync(0xffffffffu, v[t].lo, o);
                v[t] = ff_add(v[t], y);
            }
        }
        if (l == 0)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                red[8 * nw + 2 * t] = v[t].hi;
                red[8 * nw + 2 * t + 1] = v[t].lo;
            }
    }
    __syncthreads();
    a.J = ff{red[8 * nw], red[8 * nw + 1]};
    a.L = ff{red[8 * nw + 2], red[8 * nw + 3]};
    b.J = ff{red[8 * nw + 4], red[8 * nw + 5]};
    b.L = ff{red[8 * nw + 6], red[8 * nw + 7]};
    __syncthreads();
#endif
}

// Sum of the n column partials of one loop in a fixed order (lane l takes l, l+32, ..., then a
// shuffle tree), identical in every CTA; every lane of the calling warp gets the sums.
KS_HD void sum_partials(const double* a, const double* c, int n, double& sa, double& sc) {
    warp_sum_partials(a, c, n, sa, sc);
}

KS_HD void sum_partials(const ff* a, const ff* c, int n, double& sa, double& sc) {
#ifdef KS_HOST_EMULATION
    ff x = {0.f, 0.f}, y = {0.f, 0.f};
    for (int i = 0; i < n; ++i) {
        x = ff_add(x, a[i]);
        y = ff_add(y, c[i]);
    }
    sa = widen(x);
    sc = widen(y);
#else
    const int l = threadIdx.x & 31;
    ff x = {0.f, 0.f}, y = {0.f, 0.f};
    for (int i = l; i < n; i += 32) {
        x = ff_add(x, a[i]);
        y = ff_add(y, c[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ff bx, by;
        bx.hi = __shfl_xor_sync(0xffffffffu, x.hi, o);
        bx.lo = __shfl_xor_sync(0xffffffffu, x.lo, o);
        by.hi = __shfl_xor_sync(0xffffffffu, y.hi, o);
        by.lo = __shfl_xor_sync(0xffffffffu, y.lo, o);
        x = ff_add(x, bx);
        y = ff_add(y, by);
    }
    sa = widen(x);
    sc = widen(y);
#endif
}

// The freeze decision of a loop after the reductions of a step (J and the current T): diverged
// (J not finite or huge, T not positive), converged (sqrt(J) < tol), the float phase's switch
// threshold reached, or running.  Taken by one thread of a column item, which passes the int on
// through shared memory: in double, a compare occupies the FP64 pipe for a whole warp-issue slot.
template <typename R>
KS_HD int freeze_status(const Bufs<R>& p, double J, double T) {
    if (!(J == J) || J > 1e300 || !(T > 0.0)) return ST_DIVERGED;
    if (J < p.tol * p.tol) return ST_CONVERGED;
    if (p.myprec == 1 && p.switch_tol > 0.0 && J <= p.switch_tol * p.switch_tol) return ST_SWITCH;
    return ST_RUNNING;
}

// 1 / (2 pi), for L^dag_2 = (L / T^2) 2 pi S = L (2 pi / T)^2 S / (2 pi) from the stored 2 pi / T
constexpr double kInv2Pi = 0.5 / 3.14159265358979323846;

// The scalars of loop b's tau-step once its column partials are complete: J and L^dag_2 (the
// partials summed in a fixed order, as every launch form sums them), the freeze decision, sqrt(J)
// and, at step parity par ^ 1, the next T by explicit Euler (Sec. 4.2) and 2 pi / T, or the
// current ones carried forward with the status when the loop freezes.  Per loop, not per column:
// one warp of the ROW_ADJ item that holds the loop's first rows calls it, so the COL_UPDATE items
// of the loop find the decision in p.status instead of each forming it again.
template <typename R>
KS_HD void loop_scalars(const Dims& d, const Bufs<R>& p, int b, int par) {
    const int B = d.B, nkx = d.nkx;
    double sJ, sL;
    sum_partials(p.Jpart + (size_t)b * nkx, p.L2part + (size_t)b * nkx, nkx, sJ, sL);
    if ((KS_TID & 31) == 0) {
        const double T = p.T[(size_t)par * B + b], wT = p.wT[(size_t)par * B + b];
        const double J = sJ * d.L;
        // (L / T^2) 2 pi sum, with 2 pi / T^2 = (2 pi / T)^2 / (2 pi): no division
        const double L2 = sL * d.L * (wT * wT) * kInv2Pi;
        const int st = freeze_status(p, J, T);
        double* Tn = p.T + (size_t)(par ^ 1) * B;
        double* wTn = p.wT + (size_t)(par ^ 1) * B;
        p.sqrtJ[b] = sqrt(J);
        if (st != ST_RUNNING) {
            p.status[b] = st;
            Tn[b] = T;
            wTn[b] = wT;
        } else {
            const double Tnew = T - d.dtau * L2;  // explicit Euler for T (Sec. 4.2)
            Tn[b] = Tnew;
            wTn[b] = 2.0 * 3.14159265358979323846 / Tnew;
            p.steps[b] += 1;
        }
    }
}

// is the loop processed by this kernel set?
template <typename R>
KS_HD bool loop_live(const Bufs<R>& p, int b) {
    if (!p.check_active) return true;
    return p.prec[b] == p.myprec && p.status[b] == ST_RUNNING;
}

// ---- centre-symmetric (Xi) subspace: the rows of u and u_x in pairs -------------------------
// In the subspace every grid row of u is odd in x and its x-derivative u_x is even, so two rows
// a, b share one complex x-transform: y = (u_a + i u_b) + (u_x,a + i u_x,b), whose odd part in x
// is u_a + i u_b and whose even part is u_x,a + i u_x,b.  Its spectrum at x-mode J (signed
// wavenumber q_J) is Y(J) = (1 + i q_J) (U_a(J) + i U_b(J)), U(J) the rows' spectra (the mixed
// value v_j for J = j <= Kx, its conjugate for J = Nx - j).  One transform per row pair replaces
// the transform of u + i u_x per row.
template <typename R>
KS_HD cpx<R> xi_zpair(cpx<R> ua, cpx<R> ub, R qJ) {
    const cpx<R> c = mk<R>(ua.x - ub.y, ua.y + ub.x);  // U_a + i U_b
    return mk<R>(c.x - qJ * c.y, c.y + qJ * c.x);      // (1 + i q_J) c
}

// The rows from y[m] and y[-m]: u = odd part, u_x = even part.
template <typename R>
KS_HD void xi_zsplit(cpx<R> ym, cpx<R> yn, R& ua, R& ub, R& uxa, R& uxb) {
    ua = (R)0.5 * (ym.x - yn.x);
    ub = (R)0.5 * (ym.y - yn.y);
    uxa = (R)0.5 * (ym.x + yn.x);
    uxb = (R)0.5 * (ym.y + yn.y);
}

// ------------------------------------------------------------------------------------
// Row items (x-direction work on a tile of rows of one loop)
// ------------------------------------------------------------------------------------
enum RowMode { ROW_ANALYZE = 0, ROW_NONLIN = 1, ROW_ADJ = 2, ROW_SYNTH = 3 };

// Fill A[pair][J] (J in [0, Nx), row-skewed) with the Hermitian-extended spectra of two rows
// (a = 2*pair, b = 2*pair + 1) read from M: Z_J = X^a_J + i X^b_J with X_{-j} = conj(X_j).
template <typename R>
KS_HD void load_pair_spectra(const Dims& d, const cpx<R>* Mb, int ns, int n0, int lgp,
                             cpx<R>* A) {
    const int nx = d.nx, kx = d.kx;
    const int npairs = 1 << lgp;
    const int total = nx << lgp;
    for (int i = KS_TID; i < total; i += KS_NT) {
        const int J = i >> lgp;
        const int pr = i & (npairs - 1);
        cpx<R> z = mk<R>(0, 0);
        int j = -1;
        bool neg = false;
        if (J <= kx) {
            j = J;
        } else if (J >= nx - kx) {
            j = nx - J;
            neg = true;
        }
        if (j >= 0) {
            const cpx<R>* col = Mb + (size_t)j * ns + n0 + 2 * pr;
            cpx<R> xa = col[0], xb = col[1];
            if (neg) {
                xa = conj(xa);
                xb = conj(xb);
            }
            z = xa + mul_i(xb, 1);
        }
        A[(size_t)pr * nx + (J ^ row_skew<R>(pr, nx))] = z;  // row-skewed (the transform's SKI)
    }
}

// From Y = FFT(y_a + i y_b) (forward, unscaled, row-skewed) extract the half spectra of the two
// real rows,
// scaled by 1/Nx, for j = 0..Kx, and store them to M[j][n0 + 2 pr + {0,1}].
template <typename R>
KS_HD void store_pair_spectra(const Dims& d, const cpx<R>* Y, cpx<R>* Mb, int ns, int n0,
                              int lgp) {
    const int nx = d.nx;
    const R h = (R)d.hx;
    const int npairs = 1 << lgp;
    const int total = d.nkx << lgp;
    for (int i = KS_TID; i < total; i += KS_NT) {
        const int j = i >> lgp;
        const int pr = i & (npairs - 1);
        const int sk = row_skew<R>(pr, nx);  // Y is row-skewed (the transform's SKO)
        const cpx<R> yj = Y[(size_t)pr * nx + (j ^ sk)];
        const cpx<R> ym = conj(Y[(size_t)pr * nx + (((nx - j) & (nx - 1)) ^ sk)]);
        const cpx<R> sm = yj + ym;  // 2 X^a
        const cpx<R> df = yj - ym;  // 2 i X^b
        cpx<R>* col = Mb + (size_t)j * ns + n0 + 2 * pr;
        col[0] = scale(sm, h);
        col[1] = mk<R>(df.y * h, -df.x * h);
    }
}

// SWZ: p.tw is the bank-swizzled shared-memory copy of the twiddle table (load_twiddles).
// par: step parity of the T arrays (the persistent kernel passes its step's; the per-phase
// launches take p.par).
template <typename R, int MODE, bool SWZ = false>
KS_HD void row_item(const Dims& d, const Bufs<R>& p, int item, unsigned char* smem, int par = -1) {
    const RowItem it = p.rows[item];
    const int b = it.b;
    if constexpr (MODE == ROW_NONLIN || MODE == ROW_ADJ) {
        if (!loop_live(p, b)) return;
    }
    const int nx = d.nx, lgnx = d.lgnx, kx = d.kx;
    const int ns = p.ns[b];
    const int n0 = it.n0, nr = it.nr, lgnr = it.lgnr;
    const int lgp = lgnr - 1, npairs = nr >> 1;
    cpx<R>* A = reinterpret_cast<cpx<R>*>(smem);
    cpx<R>* Bf = A + (size_t)nr * nx;
    cpx<R>* Mb = p.M + p.moff[b];
    R* Ub = p.U + p.goff[b];
    R* Ib = p.io ? p.io + p.goff[b] : nullptr;

    if constexpr (MODE == ROW_ANALYZE) {
        // y = u_a + i u_b for each row pair, forward transform, split
        const int total = npairs * nx;
        for (int i = KS_TID; i < total; i += KS_NT) {
            const int pr = i >> lgnx;
            const int m = i & (nx - 1);
            const R* ra = Ib + (size_t)(n0 + 2 * pr) * nx;
            A[i] = mk<R>(ra[m], ra[nx + m]);
        }
        KS_SYNC();
        cpx<R>* Y = fft_pair<R, SWZ, false, true>(A, Bf, lgnx, npairs, -1, p.tw, 0, p.twsh);
        store_pair_spectra(d, Y, Mb, ns, n0, lgp);
        KS_SYNC();
    } else if constexpr (MODE == ROW_SYNTH) {
        load_pair_spectra(d, Mb, ns, n0, lgp, A);
        KS_SYNC();
        cpx<R>* z = fft_pair<R, SWZ, true, false>(A, Bf, lgnx, npairs, +1, p.tw, 0, p.twsh);
        const int total = npairs * nx;
        for (int i = KS_TID; i < total; i += KS_NT) {
            const int pr = i >> lgnx;
            const int m = i & (nx - 1);
            R* ra = Ib + (size_t)(n0 + 2 * pr) * nx;
            ra[m] = z[i].x;
            ra[nx + m] = z[i].y;
        }
        KS_SYNC();
    } else if constexpr (MODE == ROW_NONLIN) {
        if (p.xi) {
            // centre-symmetric subspace: u and u_x of a row pair in one transform (xi_zpair)
            const int total = npairs * nx;
            for (int i = KS_TID; i < total; i += KS_NT) {
                const int J = i >> lgp;
                const int pr = i & (npairs - 1);
                cpx<R> y = mk<R>(0, 0);
                if (J <= kx) {
                    const cpx<R>* col = Mb + (size_t)J * ns + n0 + 2 * pr;
                    y = xi_zpair(col[0], col[1], p.qv[J]);
                } else if (J >= nx - kx) {
                    const cpx<R>* col = Mb + (size_t)(nx - J) * ns + n0 + 2 * pr;
                    y = xi_zpair(conj(col[0]), conj(col[1]), -p.qv[nx - J]);
                }
                A[(size_t)pr * nx + (J ^ row_skew<R>(pr, nx))] = y;
            }
            KS_SYNC();
            cpx<R>* yv = fft_pair<R, SWZ, true, false>(A, Bf, lgnx, npairs, +1, p.tw, 0, p.twsh);
            cpx<R>* Y = (yv == A) ? Bf : A;
            for (int i = KS_TID; i < total; i += KS_NT) {
                const int pr = i >> lgnx;
                const int m = i & (nx - 1);
                R ua, ub, uxa, uxb;
                xi_zsplit(yv[i], yv[(size_t)pr * nx + ((nx - m) & (nx - 1))], ua, ub, uxa, uxb);
                R* urow = Ub + (size_t)(n0 + 2 * pr) * nx;
                urow[m] = ua;
                urow[nx + m] = ub;
                Y[i] = mk<R>(ua * uxa, ub * uxb);
            }
            KS_SYNC();
            cpx<R>* F = fft_pair<R, SWZ, false, true>(Y, yv, lgnx, npairs, -1, p.tw, 0, p.twsh);  // a4 (x-pass)
            store_pair_spectra(d, F, Mb, ns, n0, lgp);
            KS_SYNC();
            return;
        }
        // z = u + i u_x per row: Z_j = (1 - q_j) v_j, Z_{-j} = (1 + q_j) conj(v_j)   (a1, a2)
        const int total = nr * nx;
        for (int i = KS_TID; i < total; i += KS_NT) {
            const int J = i >> lgnr;
            const int r = i & (nr - 1);
            cpx<R> z = mk<R>(0, 0);
            if (J <= kx) {
                z = scale(Mb[(size_t)J * ns + n0 + r], (R)1 - p.qv[J]);
            } else if (J >= nx - kx) {
                const int j = nx - J;
                z = scale(conj(Mb[(size_t)j * ns + n0 + r]), (R)1 + p.qv[j]);
            }
            A[(size_t)r * nx + (J ^ row_skew<R>(r, nx))] = z;
        }
        KS_SYNC();
        cpx<R>* z = fft_batch<R, SWZ, true, false>(A, Bf, lgnx, nr, +1, p.tw, 0, p.twsh);
        cpx<R>* Y = (z == A) ? Bf : A;
        // keep u, form p = u u_x for the row pairs (a3)
        const int tp = npairs * nx;
        for (int i = KS_TID; i < tp; i += KS_NT) {
            const int pr = i >> lgnx;
            const int m = i & (nx - 1);
            const cpx<R> za = z[(size_t)(2 * pr) * nx + m];
            const cpx<R> zb = z[(size_t)(2 * pr + 1) * nx + m];
            R* ua = Ub + (size_t)(n0 + 2 * pr) * nx;
            ua[m] = za.x;
            ua[nx + m] = zb.x;
            Y[i] = mk<R>(za.x * za.y, zb.x * zb.y);
        }
        KS_SYNC();
        cpx<R>* F = fft_pair<R, SWZ, false, true>(Y, z, lgnx, npairs, -1, p.tw, 0, p.twsh);  // a4 (x-pass)
        store_pair_spectra(d, F, Mb, ns, n0, lgp);
        KS_SYNC();
    } else if constexpr (MODE == ROW_ADJ) {
        // r_x rows from the column pass output rho = s-inverse of i q_j r_hat   (a7)
        load_pair_spectra(d, Mb, ns, n0, lgp, A);
        KS_SYNC();
        cpx<R>* z = fft_pair<R, SWZ, true, false>(A, Bf, lgnx, npairs, +1, p.tw, 0, p.twsh);
        cpx<R>* Y = (z == A) ? Bf : A;
        const int tp = npairs * nx;
        for (int i = KS_TID; i < tp; i += KS_NT) {
            const int pr = i >> lgnx;
            const int m = i & (nx - 1);
            const R* ua = Ub + (size_t)(n0 + 2 * pr) * nx;
            const cpx<R> rx = z[i];
            Y[i] = mk<R>(ua[m] * rx.x, ua[nx + m] * rx.y);  // w = u r_x  (a8)
        }
        KS_SYNC();
        cpx<R>* F = fft_pair<R, SWZ, false, true>(Y, z, lgnx, npairs, -1, p.tw, 0, p.twsh);
        store_pair_spectra(d, F, Mb, ns, n0, lgp);
        KS_SYNC();
        // double: the loop's step scalars, once per loop (the column partials are complete since
        // COL_RESID), after the item's last barrier so the rest of the block moves on; float:
        // after the launch's items (loops_scalars)
        if constexpr (sizeof(R) == 8) {
            if (p.step_scalars && n0 == 0 && KS_TID < 32) loop_scalars(d, p, b, par < 0 ? p.par : par);
        }
    }
}

// Float: the step scalars of every live loop (loop_scalars), loop b on block b mod nblk, its
// first warp.  The launches that run the ROW_ADJ items call it after them: the column partials
// are complete since COL_RESID, and the ROW_ADJ items do not read T.  Called inside an item it
// raised the float kernel's registers from 32 to 48 (10 instead of 16 resident blocks of 128
// threads); outside the item loop it takes 36, and the per-phase float step got 2-4 % faster
// (ragged256 82.7 -> 79.7 us, large8_256x1024 75.9 -> 74.2 us).  The double kernel keeps the call
// in the item: outside it ptxas held the kernel to 32 registers with a spill, and the 256x1024
// double step got 2 % slower.  Same arithmetic either way.
template <typename R>
KS_HD void loops_scalars(const Dims& d, const Bufs<R>& p, int par, int blk, int nblk) {
    if constexpr (sizeof(R) == 8) return;
    if (!p.step_scalars || KS_TID >= 32) return;
    for (int b = blk; b < d.B; b += nblk)
        if (loop_live(p, b)) loop_scalars(d, p, b, par);
}

// ------------------------------------------------------------------------------------
// Column items (s-direction work on one retained x-mode j of one loop)
// ------------------------------------------------------------------------------------
enum ColMode {
    COL_ANALYZE = 0,  // M -> band u_hat (forward, 1/Ns, truncate)
    COL_SYNTH_U = 1,  // band u_hat -> M (inverse)
    COL_SYNTH_R = 2,  // band r_hat -> M
    COL_SYNTH_G = 3,  // band G_hat -> M
    COL_RESID = 4,    // M = P -> r_hat, partials, M = s-inverse of i q r_hat
    COL_UPDATE = 5,   // M = W -> G_hat, update u_hat and T, M = s-inverse of new u_hat
    COL_GRAD = 6      // M = W -> G_hat band (no update)
};

// Shared-memory bytes a column item needs beyond its two transform buffers.
constexpr int COL_RED_DOUBLES = 4 * (256 / 32 + 1) + 4;  // blocks of up to 256 threads


// Threads that accumulate one column's J and L^dag_2 partial: element n of a column goes to
// accumulator n mod COL_ACC_LANES in every launch form, whatever the block size, so the partial
// (and everything downstream of it) is the same bits in the item kernels (128 threads) and in a
// cluster kernel of 128 or 256 threads.
constexpr int COL_ACC_LANES = 128;

// A column item of more than COL_ACC_LANES threads forms r_hat with all of them, then its first
// COL_ACC_LANES threads accumulate the column from the stored band (the same values in the same
// order per accumulator); with exactly COL_ACC_LANES threads the accumulation is fused into the
// loop that forms r_hat.
#ifdef KS_HOST_EMULATION
#define KS_ACC_FUSED true
#else
#define KS_ACC_FUSED ((int)blockDim.x == COL_ACC_LANES)
#endif

// ---- centre-symmetric (Xi) subspace: columns in pairs --------------------------------------
// In the subspace u_hat_{j,-k} = -conj(u_hat_{j,k}) and the j = 0 column is zero, so the s-series
// of every retained x-mode j >= 1 is purely imaginary (u, the products u u_x and u r_x, all odd
// in x) or purely real (r_x, even in x).  Two such columns share one complex s-transform: the
// canonical pairs are (2p + 1, 2p + 2), p = 0 .. ceil(Kx / 2) - 1, the second column absent when
// 2p + 2 > Kx.  Forward, of imaginary columns x_a = i xi_a, x_b = i xi_b: C = F[xi_a + i xi_b],
// X_a(k) = i (C(k) + conj C(-k)) / 2, X_b(k) = (C(k) - conj C(-k)) / 2.  Inverse to imaginary
// columns: c = F^-1[-i X_a + X_b], x_a = i Re c, x_b = i Im c; to real columns:
// c = F^-1[X_a + i X_b], x_a = Re c, x_b = Im c.  The split gives X(-k) = -conj X(k) bit for bit
// (IEEE negation is exact, addition commutes), so the band keeps the subspace's symmetry exactly
// without a projection, and the x-mode j = 0 needs no transform at all.  Every launch form pairs
// the same columns, so they compute the same bits.
KS_HDX int xi_npairs(const Dims& d) { return (d.kx + 1) / 2; }

// the column modes that run on pairs in the subspace
KS_HDX constexpr bool col_paired(int MODE) {
    return MODE == COL_SYNTH_U || MODE == COL_RESID || MODE == COL_UPDATE || MODE == COL_GRAD;
}

// number of work items of a column phase
KS_HDX int col_item_count(const Dims& d, int xi, int MODE) {
    return d.B * ((xi && col_paired(MODE)) ? xi_npairs(d) : d.nkx);
}

template <typename R>
KS_HD cpx<R> xi_split_a(cpx<R> ck, cpx<R> cm) {  // X_a(k) from C(k), C(-k)
    return mk<R>((R)0.5 * (cm.y - ck.y), (R)0.5 * (ck.x + cm.x));
}
template <typename R>
KS_HD cpx<R> xi_split_b(cpx<R> ck, cpx<R> cm) {  // X_b(k)
    return mk<R>((R)0.5 * (ck.x - cm.x), (R)0.5 * (ck.y + cm.y));
}
template <typename R>
KS_HD cpx<R> xi_join_imag(cpx<R> xa, cpx<R> xb) {  // -i X_a + X_b
    return mk<R>(xa.y + xb.x, xb.y - xa.x);
}
template <typename R>
KS_HD cpx<R> xi_join_real(cpx<R> xa, cpx<R> xb) {  // X_a + i X_b
    return mk<R>(xa.x - xb.y, xa.y + xb.x);
}
template <typename P>
KS_HD P zero_part() { return P{}; }

// One pair of columns (ja, jb) of one loop; the modes of col_item that run on pairs.  Pair 0
// also writes the zero column j = 0 (M and the partials) and takes the per-loop duties that
// column 0 has in col_item (T, status, sqrt(J), the step counter).
template <typename R, int MODE, bool SWZ = false>
KS_HD void col_pair_item(const Dims& d, const Bufs<R>& p, int item, unsigned char* smem, int par) {
    typedef typename PartT<R>::type Part;
    const int nkx = d.nkx, np = xi_npairs(d);
    const int b = p.colorder[item / np];
    const int pp = item - (item / np) * np;
    const int ja = 2 * pp + 1, jb = 2 * pp + 2;
    const bool hasb = jb <= d.kx;
    const int ns = p.ns[b], lg = p.lgns[b], ks = p.ks[b];
    const int nk = 2 * ks + 1;
    cpx<R>* A = reinterpret_cast<cpx<R>*>(smem);
    cpx<R>* Bf = A + ns;
    double* red = reinterpret_cast<double*>(Bf + ns);
    cpx<R>* const M0 = p.M + p.moff[b];
    cpx<R>* const cola = M0 + (size_t)ja * ns;
    cpx<R>* const colb = M0 + (size_t)jb * ns;   // used only when hasb
    const size_t ba = (size_t)p.boff[b] + (size_t)ja * nk;
    const size_t bb = (size_t)p.boff[b] + (size_t)jb * nk;
    const int B = d.B;
    const double* Tc = p.T + (size_t)par * B;
    double* Tn = p.T + (size_t)(par ^ 1) * B;
    const double* wTc = p.wT + (size_t)par * B;
    double* wTn = p.wT + (size_t)(par ^ 1) * B;
    const cpx<R> zero = mk<R>(0, 0);

    if constexpr (MODE == COL_RESID || MODE == COL_GRAD) {
        if (!loop_live(p, b)) return;
    }
    if constexpr (MODE == COL_UPDATE) {
        if (p.check_active && p.prec[b] != p.myprec) return;
        if (p.check_active && p.status[b] != ST_RUNNING) {
            if (pp == 0 && KS_TID == 0) {
                Tn[b] = Tc[b];
                wTn[b] = wTc[b];
            }
            return;
        }
    }

    if constexpr (MODE == COL_SYNTH_U) {
        for (int i = KS_TID; i < ns; i += KS_NT) {
            const int k = (i < (ns >> 1)) ? i : i - ns;
            cpx<R> x = zero;
            if (k >= -ks && k <= ks) x = xi_join_imag(p.uh[ba + (k + ks)], hasb ? p.uh[bb + (k + ks)] : zero);
            A[i] = x;
        }
        KS_SYNC();
        const cpx<R>* v = fft_col<R, SWZ>(A, Bf, lg, 1, +1, p.tw, 0, p.twsh);
        for (int i = KS_TID; i < ns; i += KS_NT) {
            cola[i] = mk<R>(0, v[i].x);
            if (hasb) colb[i] = mk<R>(0, v[i].y);
            if (pp == 0) M0[i] = zero;
        }
        KS_SYNC();
    } else {

        // RESID, UPDATE, GRAD: forward s-transform of the imaginary columns P or W of M, in one
        for (int i = KS_TID; i < ns; i += KS_NT) A[i] = mk<R>(cola[i].y, hasb ? colb[i].y : (R)0);
        KS_SYNC();
        cpx<R>* F = fft_col<R, SWZ>(A, Bf, lg, 1, -1, p.tw, 0, p.twsh);
        cpx<R>* X = (F == A) ? Bf : A;
        const R ins = p.insv[b];
        const R w_over_T = (R)wTc[b];
        const R lin_a = p.lin[ja], lin_b = hasb ? p.lin[jb] : (R)0;
        const R q_a = p.qv[ja], q_b = hasb ? p.qv[jb] : (R)0;

        if constexpr (MODE == COL_RESID) {
            ColAcc<R> acc[2];
            const bool fused = KS_ACC_FUSED;
            for (int i = KS_TID; i < ns; i += KS_NT) {
                const int k = (i < (ns >> 1)) ? i : i - ns;
                cpx<R> x = zero;
                if (k >= -ks && k <= ks) {
                    const cpx<R> ck = F[i], cm = F[(ns - i) & (ns - 1)];
                    const R bk = -(R)k * w_over_T;            // -omega_k / T
                    // r_hat = (a + i bk) u_hat - p_hat for both columns                     (a5)
                    const cpx<R> pa = scale(xi_split_a(ck, cm), ins);
                    const cpx<R> ua = p.uh[ba + (k + ks)];
                    const cpx<R> ra = mk<R>(lin_a * ua.x - bk * ua.y - pa.x, lin_a * ua.y + bk * ua.x - pa.y);
                    p.rh[ba + (k + ks)] = ra;
                    if (fused) acc[0].add(ua, ra, k);         // a6
                    cpx<R> xb = zero;
                    if (hasb) {
                        const cpx<R> pb = scale(xi_split_b(ck, cm), ins);
                        const cpx<R> ub = p.uh[bb + (k + ks)];
                        const cpx<R> rb = mk<R>(lin_b * ub.x - bk * ub.y - pb.x, lin_b * ub.y + bk * ub.x - pb.y);
                        p.rh[bb + (k + ks)] = rb;
                        if (fused) acc[1].add(ub, rb, k);
                        xb = mk<R>(-q_b * rb.y, q_b * rb.x);   // i q_j r_hat                 (a7)
                    }
                    x = xi_join_real(mk<R>(-q_a * ra.y, q_a * ra.x), xb);
                }
                X[i] = x;
            }
            KS_SYNC();
            if (!fused && KS_TID < COL_ACC_LANES)
                for (int i = KS_TID; i < ns; i += COL_ACC_LANES) {
                    const int k = (i < (ns >> 1)) ? i : i - ns;
                    if (k >= -ks && k <= ks) {
                        acc[0].add(p.uh[ba + (k + ks)], p.rh[ba + (k + ks)], k);
                        if (hasb) acc[1].add(p.uh[bb + (k + ks)], p.rh[bb + (k + ks)], k);
                    }
                }
            const cpx<R>* v = fft_col<R, SWZ>(X, F, lg, 1, +1, p.tw, 0, p.twsh);
            for (int i = KS_TID; i < ns; i += KS_NT) {
                cola[i] = mk<R>(v[i].x, 0);
                if (hasb) colb[i] = mk<R>(v[i].y, 0);
                if (pp == 0) M0[i] = zero;
            }
            block_reduce2(acc[0], acc[1], red);
            if (KS_TID == 0) {
                p.Jpart[(size_t)b * nkx + ja] = acc[0].part_J(2.0);
                p.L2part[(size_t)b * nkx + ja] = acc[0].part_L(2.0);
                if (hasb) {
                    p.Jpart[(size_t)b * nkx + jb] = acc[1].part_J(2.0);
                    p.L2part[(size_t)b * nkx + jb] = acc[1].part_L(2.0);
                }
                if (pp == 0) {
                    p.Jpart[(size_t)b * nkx] = zero_part<Part>();
                    p.L2part[(size_t)b * nkx] = zero_part<Part>();
                }
            }
            KS_SYNC();
            return;
        }

        // G_hat = (a + i omega/T) r_hat + F[P(u r_x)] for both columns at mode k              (a9)
        auto g_at = [&](int i, int k, bool second) {
            const cpx<R> ck = F[i], cm = F[(ns - i) & (ns - 1)];
            const cpx<R> wh = scale(second ? xi_split_b(ck, cm) : xi_split_a(ck, cm), ins);
            const cpx<R> r = p.rh[(second ? bb : ba) + (k + ks)];
            const R a_lin = second ? lin_b : lin_a;
            const R bk = (R)k * w_over_T;
            return mk<R>(a_lin * r.x - bk * r.y + wh.x, a_lin * r.y + bk * r.x + wh.y);
        };

        if constexpr (MODE == COL_GRAD) {
            for (int i = KS_TID; i < ns; i += KS_NT) {
                const int k = (i < (ns >> 1)) ? i : i - ns;
                if (k >= -ks && k <= ks) {
                    p.gh[ba + (k + ks)] = g_at(i, k, false);
                    if (hasb) p.gh[bb + (k + ks)] = g_at(i, k, true);
                }
            }
            if (pp == 0)  // the j = 0 column of G is zero in the subspace
                for (int kk = KS_TID; kk < nk; kk += KS_NT) p.gh[(size_t)p.boff[b] + kk] = zero;
            KS_SYNC();
            return;
        }

        if constexpr (MODE == COL_UPDATE) {
            // J, the freeze decision and the next T of this step were formed once for the loop
            // by the ROW_ADJ launch (loop_scalars): a loop that froze now is in p.status
            if (p.status[b] != ST_RUNNING) return;
            const R dt = (R)d.dtau;
            const R wT2 = w_over_T * w_over_T;
            const R cq_a = p.cq[ja], cq_b = hasb ? p.cq[jb] : (R)0;
            for (int i = KS_TID; i < ns; i += KS_NT) {
                const int k = (i < (ns >> 1)) ? i : i - ns;
                cpx<R> x = zero;
                if (k >= -ks && k <= ks) {
                    R fa = dt, fb = dt;
                    if (d.scheme == 1) {
                        // IMEX: dtau / (1 - dtau Lambda), Lambda = -(omega/T)^2 - q^4 (q^2-1)^2  (a10)
                        const R kk2 = (R)k * (R)k;
                        fa = dt / ((R)1 + dt * (kk2 * wT2 + cq_a));
                        fb = dt / ((R)1 + dt * (kk2 * wT2 + cq_b));
                    }
                    cpx<R> ua = p.uh[ba + (k + ks)];
                    ua = ua - scale(g_at(i, k, false), fa);
                    p.uh[ba + (k + ks)] = ua;
                    cpx<R> ub = zero;
                    if (hasb) {
                        ub = p.uh[bb + (k + ks)];
                        ub = ub - scale(g_at(i, k, true), fb);
                        p.uh[bb + (k + ks)] = ub;
                    }
                    x = xi_join_imag(ua, ub);
                }
                X[i] = x;
            }
            KS_SYNC();
            const cpx<R>* v = fft_col<R, SWZ>(X, F, lg, 1, +1, p.tw, 0, p.twsh);
            for (int i = KS_TID; i < ns; i += KS_NT) {
                cola[i] = mk<R>(0, v[i].x);
                if (hasb) colb[i] = mk<R>(0, v[i].y);
                if (pp == 0) M0[i] = zero;
            }
            KS_SYNC();
        }
    }
}

template <typename R, int MODE, bool SWZ = false>
KS_HD void col_item(const Dims& d, const Bufs<R>& p, int item, unsigned char* smem, int par) {
    if constexpr (col_paired(MODE)) {
        if (p.xi) {
            col_pair_item<R, MODE, SWZ>(d, p, item, smem, par);
            return;
        }
    }
    const int nkx = d.nkx;
    const int b = p.colorder[item / nkx];
    const int j = item - (item / nkx) * nkx;
    const int ns = p.ns[b], lg = p.lgns[b], ks = p.ks[b];
    const int nk = 2 * ks + 1;
    cpx<R>* A = reinterpret_cast<cpx<R>*>(smem);
    cpx<R>* Bf = A + ns;
    double* red = reinterpret_cast<double*>(Bf + ns);
    cpx<R>* col = p.M + p.moff[b] + (size_t)j * ns;
    const size_t bo = (size_t)p.boff[b] + (size_t)j * nk;
    const int B = d.B;
    const double* Tc = p.T + (size_t)par * B;
    double* Tn = p.T + (size_t)(par ^ 1) * B;
    const double* wTc = p.wT + (size_t)par * B;
    double* wTn = p.wT + (size_t)(par ^ 1) * B;

    if constexpr (MODE == COL_RESID || MODE == COL_GRAD) {
        if (!loop_live(p, b)) return;
    }
    if constexpr (MODE == COL_UPDATE) {
        if (p.check_active && p.prec[b] != p.myprec) return;
        if (p.check_active && p.status[b] != ST_RUNNING) {
            if (j == 0 && KS_TID == 0) {
                Tn[b] = Tc[b];
                wTn[b] = wTc[b];
            }
            return;
        }
    }

    if constexpr (MODE == COL_SYNTH_U || MODE == COL_SYNTH_R || MODE == COL_SYNTH_G) {
        const cpx<R>* src = (MODE == COL_SYNTH_U) ? p.uh : (MODE == COL_SYNTH_R) ? p.rh : p.gh;
        for (int i = KS_TID; i < ns; i += KS_NT) {
            const int k = (i < (ns >> 1)) ? i : i - ns;
            A[i] = (k >= -ks && k <= ks) ? src[bo + (k + ks)] : mk<R>(0, 0);
        }
        KS_SYNC();
        cpx<R>* v = fft_col<R, SWZ>(A, Bf, lg, 1, +1, p.tw, 0, p.twsh);
        for (int i = KS_TID; i < ns; i += KS_NT) col[i] = v[i];
        KS_SYNC();
    } else {
        // the remaining modes start with a forward s-transform of the column of M
        for (int i = KS_TID; i < ns; i += KS_NT) A[i] = col[i];
        KS_SYNC();
        cpx<R>* F = fft_col<R, SWZ>(A, Bf, lg, 1, -1, p.tw, 0, p.twsh);
        cpx<R>* X = (F == A) ? Bf : A;
        const R ins = p.insv[b];

        if constexpr (MODE == COL_ANALYZE) {
            for (int kk = KS_TID; kk < nk; kk += KS_NT) {
                const int k = kk - ks;
                cpx<R> v = scale(F[k & (ns - 1)], ins);
                if (p.xi) v = (j == 0) ? mk<R>(0, 0) : xi_pair(v, scale(F[(-k) & (ns - 1)], ins));
                p.uh[bo + kk] = v;
            }
            KS_SYNC();
            return;
        }

        const R a_lin = p.lin[j];       // q^2 - q^4 (from -u_xx - u_xxxx)
        const R w_over_T = (R)wTc[b];   // omega_k / T = k * (2 pi / T)
        const R rq = p.qv[j];
        const double wj = (j == 0) ? 1.0 : 2.0;  // x-conjugate pairs counted twice

        if constexpr (MODE == COL_RESID) {
            ColAcc<R> acc;
            const bool fused = KS_ACC_FUSED;
            for (int i = KS_TID; i < ns; i += KS_NT) {
                const int k = (i < (ns >> 1)) ? i : i - ns;
                cpx<R> x = mk<R>(0, 0);
                if (k >= -ks && k <= ks) {
                    const cpx<R> ph = scale(F[i], ins);
                    const cpx<R> u = p.uh[bo + (k + ks)];
                    const R bk = -(R)k * w_over_T;            // -omega_k / T
                    // r_hat = (a + i bk) u_hat - p_hat                                    (a5)
                    const cpx<R> r = mk<R>(a_lin * u.x - bk * u.y - ph.x, a_lin * u.y + bk * u.x - ph.y);
                    p.rh[bo + (k + ks)] = r;
                    if (fused) acc.add(u, r, k);              // a6: |r|^2, k Im(conj(u) r)
                    x = mk<R>(-rq * r.y, rq * r.x);           // i q_j r_hat                 (a7)
                }
                X[i] = x;
            }
            KS_SYNC();
            if (!fused && KS_TID < COL_ACC_LANES)
                for (int i = KS_TID; i < ns; i += COL_ACC_LANES) {
                    const int k = (i < (ns >> 1)) ? i : i - ns;
                    if (k >= -ks && k <= ks) acc.add(p.uh[bo + (k + ks)], p.rh[bo + (k + ks)], k);
                }
            cpx<R>* v = fft_col<R, SWZ>(X, F, lg, 1, +1, p.tw, 0, p.twsh);
            for (int i = KS_TID; i < ns; i += KS_NT) col[i] = v[i];
            block_reduce(acc, red);
            if (KS_TID == 0) {
                p.Jpart[(size_t)b * nkx + j] = acc.part_J(wj);
                p.L2part[(size_t)b * nkx + j] = acc.part_L(wj);
            }
            KS_SYNC();
        } else if constexpr (MODE == COL_GRAD) {
            for (int i = KS_TID; i < ns; i += KS_NT) {
                const int k = (i < (ns >> 1)) ? i : i - ns;
                if (k >= -ks && k <= ks) {
                    const cpx<R> wh = scale(F[i], ins);
                    const cpx<R> r = p.rh[bo + (k + ks)];
                    const R bk = (R)k * w_over_T;             // +omega_k / T
                    const cpx<R> G = mk<R>(a_lin * r.x - bk * r.y + wh.x, a_lin * r.y + bk * r.x + wh.y);
                    if (p.xi) X[i] = G;
                    else p.gh[bo + (k + ks)] = G;
                }
            }
            KS_SYNC();
            if (p.xi) {
                // gradient within the Xi subspace: the projected G_hat
                for (int i = KS_TID; i < ns; i += KS_NT) {
                    const int k = (i < (ns >> 1)) ? i : i - ns;
                    if (k >= -ks && k <= ks)
                        p.gh[bo + (k + ks)] = (j == 0) ? mk<R>(0, 0) : xi_pair(X[i], X[(ns - i) & (ns - 1)]);
                }
                KS_SYNC();
            }
        } else if constexpr (MODE == COL_UPDATE) {
            // J, the freeze decision and the next T of this step were formed once for the loop
            // by the ROW_ADJ launch (loop_scalars): a loop that froze now is in p.status
            if (p.status[b] != ST_RUNNING) return;
            const R dt = (R)d.dtau;
            const R cqj = p.cq[j];
            const R wT2 = w_over_T * w_over_T;
            if (p.xi) {
                // Xi subspace: G_hat of every k into X first; the update below takes the
                // projected pair (j, k), (j, -k) from there
                for (int i = KS_TID; i < ns; i += KS_NT) {
                    const int k = (i < (ns >> 1)) ? i : i - ns;
                    if (k >= -ks && k <= ks) {
                        const cpx<R> wh = scale(F[i], ins);
                        const cpx<R> r = p.rh[bo + (k + ks)];
                        const R bk = (R)k * w_over_T;
                        X[i] = mk<R>(a_lin * r.x - bk * r.y + wh.x, a_lin * r.y + bk * r.x + wh.y);
                    }
                }
                KS_SYNC();
            }
            // the new u_hat goes to X, or to F (free once G_hat is formed) in the Xi subspace
            cpx<R>* Y = p.xi ? F : X;
            for (int i = KS_TID; i < ns; i += KS_NT) {
                const int k = (i < (ns >> 1)) ? i : i - ns;
                cpx<R> x = mk<R>(0, 0);
                if (k >= -ks && k <= ks) {
                    cpx<R> G;
                    if (p.xi) {
                        G = (j == 0) ? mk<R>(0, 0) : xi_pair(X[i], X[(ns - i) & (ns - 1)]);
                    } else {
                        const cpx<R> wh = scale(F[i], ins);
                        const cpx<R> r = p.rh[bo + (k + ks)];
                        const R bk = (R)k * w_over_T;
                        // G_hat = (a + i omega/T) r_hat + F[P(u r_x)]                      (a9)
                        G = mk<R>(a_lin * r.x - bk * r.y + wh.x, a_lin * r.y + bk * r.x + wh.y);
                    }
                    R f = dt;
                    if (d.scheme == 1) {
                        // IMEX: dtau / (1 - dtau Lambda), Lambda = -(omega/T)^2 - q^4 (q^2-1)^2  (a10)
                        const R kk2 = (R)k * (R)k;
                        f = dt / ((R)1 + dt * (kk2 * wT2 + cqj));
                    }
                    cpx<R> u = p.uh[bo + (k + ks)];
                    u = u - scale(G, f);
                    p.uh[bo + (k + ks)] = u;
                    x = u;
                }
                Y[i] = x;
            }
            KS_SYNC();
            cpx<R>* v = fft_col<R, SWZ>(Y, p.xi ? X : F, lg, 1, +1, p.tw, 0, p.twsh);
            for (int i = KS_TID; i < ns; i += KS_NT) col[i] = v[i];
            KS_SYNC();
        }
    }
}

}  // namespace ks
