// ks_dns.cu - time integration of the KSE itself, for the initial loops (Sec. 4.3 of the paper).
//
// The paper draws its initial loops from close recurrences of a chaotic solution u(x, t) of
// u_t = -u u_x - u_xx - u_xxxx on [0, L) (Sec. 4.3).  This file integrates that equation on the
// GPU: a Fourier pseudo-spectral discretisation with Nx points, the product dealiased by the 2/3
// rule as in the descent (Sec. 4.2), and fourth-order exponential time differencing (ETDRK4,
// Cox & Matthews, J. Comput. Phys. 176, 2002), whose linear part is the exact diagonal symbol
// q_j^2 - q_j^4.  The phi-function weights are contour averages (Kassam & Trefethen, SIAM
// J. Sci. Comput. 26, 2005) computed in the kernel at launch.  A second kernel cuts a segment
// of a saved trajectory into the Ns instants of a loop by linear interpolation in time.
//
// Layout: one CTA integrates up to DNS_PAIRS_MAX pairs of trajectories for the whole run.  The
// two real fields of a pair share one complex x-transform (u_a + i u_b, and the products
// u_a^2 + i u_b^2); the state of each trajectory is its half spectrum v_j, j = 0..Kx, kept in
// shared memory with the stage values of the scheme.  Global memory is touched at the start
// (u0), at every saved instant (u and ||u||) and at the end.  The transforms take radix-2 passes
// (fft_batch_r2): an FP64 warp instruction costs the same issue time with idle lanes, and a
// radix-2 pass has twice the butterflies of a radix-4 pass at the same operation count per
// point, so a single pair keeps a whole warp busy and four pairs fill the block's four warps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ks_items.cuh"
#include "ks_loop.h"

using namespace ks;

void ks_internal_set_error(const char* msg);

namespace {

constexpr int DNS_THREADS = 128;
constexpr int DNS_PAIRS_MAX = 4;
constexpr int DNS_CONTOUR = 32;  // points on the upper half of the contour circle
constexpr int DNS_SPECS = 7;     // v, a, s (stage b then c), Nv, Na, Nb, Nc per trajectory
constexpr int DNS_COEFS = 7;     // E, E2, Q, f1, f2, f3, g per x-mode

struct DnsArgs {
    double L, dt;
    int nx, lgnx, kx, nh, batch, pairs;  // pairs per CTA
    int save_every, symmetric;
    long long nsteps, nsave;
    const double* u0;   // [batch][nx]
    double* u_saved;    // [batch][nsave][nx] or null
    double* norms;      // [batch][nsave] or null
    double* u_end;      // [batch][nx] or null
};

// shared-memory plan: twiddles, coefficients, per pair two transform buffers of nx, per
// trajectory DNS_SPECS half spectra of nh values
struct DnsPlan {
    int off_tw, off_coef, off_fft, off_spec, off_red, bytes;
};

__host__ __device__ inline DnsPlan dns_plan(int nx, int nh, int pairs) {
    DnsPlan p;
    int o = 0;
    p.off_tw = o;
    o += nx * (int)sizeof(cpx<double>);
    p.off_coef = o;
    o += DNS_COEFS * nh * (int)sizeof(double);
    o = (o + 15) & ~15;
    p.off_fft = o;
    o += 2 * pairs * nx * (int)sizeof(cpx<double>);
    p.off_spec = o;
    o += 2 * pairs * DNS_SPECS * nh * (int)sizeof(cpx<double>);
    p.off_red = o;
    o += 2 * DNS_PAIRS_MAX * (int)sizeof(double);
    p.bytes = o;
    return p;
}

// complex helpers for the contour averages (double, device)
struct cd {
    double x, y;
};
__device__ __forceinline__ cd cadd(cd a, cd b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cd cmulc(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cscal(cd a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ cd cdivc(cd a, cd b) {
    const double d = b.x * b.x + b.y * b.y;
    return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__device__ __forceinline__ cd cexpc(cd a) {
    double s, c;
    sincos(a.y, &s, &c);
    const double e = exp(a.x);
    return {e * c, e * s};
}

// ETDRK4 weights of x-mode j (Cox & Matthews), z = dt (q^2 - q^4):
//   E = e^z, E2 = e^(z/2), Q = dt (e^(z/2) - 1) / z,
//   f1 = dt (-4 - z + e^z (4 - 3z + z^2)) / z^3, f2 = dt (2 + z + e^z (z - 2)) / z^3,
//   f3 = dt (-4 - 3z - z^2 + e^z (4 - z)) / z^3,
// each evaluated as the mean of the expression over points z + r_k on a circle of radius 1 around
// z (the expressions are entire, so the mean equals the value at z without the cancellation of
// the closed forms near z = 0); for real z the mean over the upper half circle, real part, is the
// mean over the whole circle.  g = -q/2 is the factor of the nonlinear term -(u^2/2)_x.
__device__ void dns_coefficients(double* coef, int nh, double L, double dt) {
    for (int j = threadIdx.x; j < nh; j += blockDim.x) {
        const double q = 2.0 * 3.14159265358979323846 * (double)j / L;
        const double z = dt * (q * q - q * q * q * q);
        cd sQ{0, 0}, s1{0, 0}, s2{0, 0}, s3{0, 0};
        for (int k = 1; k <= DNS_CONTOUR; ++k) {
            double sr, cr;
            sincospi(((double)k - 0.5) / (double)DNS_CONTOUR, &sr, &cr);
            const cd w{z + cr, sr};
            const cd ew = cexpc(w), ew2 = cexpc(cscal(w, 0.5));
            const cd w2 = cmulc(w, w), w3 = cmulc(w2, w);
            sQ = cadd(sQ, cdivc({ew2.x - 1.0, ew2.y}, w));
            // -4 - w + e^w (4 - 3w + w^2)
            const cd a1 = cadd({-4.0 - w.x, -w.y}, cmulc(ew, {4.0 - 3.0 * w.x + w2.x, -3.0 * w.y + w2.y}));
            // 2 + w + e^w (w - 2)
            const cd a2 = cadd({2.0 + w.x, w.y}, cmulc(ew, {w.x - 2.0, w.y}));
            // -4 - 3w - w^2 + e^w (4 - w)
            const cd a3 = cadd({-4.0 - 3.0 * w.x - w2.x, -3.0 * w.y - w2.y}, cmulc(ew, {4.0 - w.x, -w.y}));
            s1 = cadd(s1, cdivc(a1, w3));
            s2 = cadd(s2, cdivc(a2, w3));
            s3 = cadd(s3, cdivc(a3, w3));
        }
        const double im = 1.0 / (double)DNS_CONTOUR;
        coef[0 * nh + j] = exp(z);
        coef[1 * nh + j] = exp(0.5 * z);
        coef[2 * nh + j] = dt * sQ.x * im;
        coef[3 * nh + j] = dt * s1.x * im;
        coef[4 * nh + j] = dt * s2.x * im;
        coef[5 * nh + j] = dt * s3.x * im;
        coef[6 * nh + j] = -0.5 * q;
    }
}

// spectrum `which` of trajectory t (t = 2 * pair + member) in the CTA's spectra block
__device__ __forceinline__ cpx<double>* spec(cpx<double>* base, int nh, int t, int which) {
    return base + ((size_t)t * DNS_SPECS + which) * nh;
}

enum { SV = 0, SA = 1, SS = 2, SNV = 3, SNA = 4, SNB = 5, SNC = 6 };

// Sum of y over the nx points of each trajectory of the CTA (component 0: member a, 1: b),
// warp w reduces trajectories w, w + warps, ...; fixed order for a given nx.
__device__ void dns_norms(const cpx<double>* Y, int nx, int ntraj, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = w; t < ntraj; t += nw) {
        const cpx<double>* y = Y + (size_t)(t >> 1) * nx;
        double s = 0.0;
        for (int m = lane; m < nx; m += 32) s += (t & 1) ? y[m].y : y[m].x;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[t] = s;
    }
}

// One evaluation for every trajectory of the CTA: the grid field of spectrum `src` (inverse
// x-transform of the pair u_a + i u_b), optionally saved, and, when dst >= 0, the nonlinear
// term N_j = -(i q_j / 2) F[u^2]_j on the retained modes (forward transform of the pair
// u_a^2 + i u_b^2, split into the two members).
__device__ void dns_eval(const DnsArgs& a, int tr0, int ntraj, cpx<double>* fftb, cpx<double>* specs,
                         const cpx<double>* tw, const double* coef, double* red, int src, int dst,
                         long long isave, bool end) {
    const int nx = a.nx, lgnx = a.lgnx, kx = a.kx, nh = a.nh;
    const int np = (ntraj + 1) >> 1;
    const int twsh = LGNMAX - lgnx;
    cpx<double>* A = fftb;
    cpx<double>* Bf = fftb + (size_t)a.pairs * nx;
    for (int i = threadIdx.x; i < np * nx; i += blockDim.x) {
        const int pr = i >> lgnx, J = i & (nx - 1);
        const int ta = 2 * pr, tb = ta + 1;
        const bool hb = tb < ntraj;
        cpx<double> z = mk<double>(0, 0);
        if (J <= kx) {
            const cpx<double> va = spec(specs, nh, ta, src)[J];
            const cpx<double> vb = hb ? spec(specs, nh, tb, src)[J] : mk<double>(0, 0);
            z = mk<double>(va.x - vb.y, va.y + vb.x);               // v_a + i v_b
        } else if (J >= nx - kx) {
            const cpx<double> va = spec(specs, nh, ta, src)[nx - J];
            const cpx<double> vb = hb ? spec(specs, nh, tb, src)[nx - J] : mk<double>(0, 0);
            z = mk<double>(va.x + vb.y, -va.y + vb.x);              // conj v_a + i conj v_b
        }
        A[i] = z;
    }
    __syncthreads();
    cpx<double>* Z = fft_batch_r2<double, true>(A, Bf, lgnx, np, +1, tw, 0, twsh);
    cpx<double>* Y = (Z == A) ? Bf : A;
    const double inx = 1.0 / (double)nx;  // exact: nx is a power of two
    const bool save = isave >= 0;
    for (int i = threadIdx.x; i < np * nx; i += blockDim.x) {
        const int pr = i >> lgnx, m = i & (nx - 1);
        const double ua = Z[i].x * inx, ub = Z[i].y * inx;
        Y[i] = mk<double>(ua * ua, ub * ub);
        if (save) {
            const int ta = tr0 + 2 * pr, tb = ta + 1;
            if (a.u_saved) {
                a.u_saved[((size_t)ta * a.nsave + isave) * nx + m] = ua;
                if (2 * pr + 1 < ntraj) a.u_saved[((size_t)tb * a.nsave + isave) * nx + m] = ub;
            }
        }
        if (end && a.u_end) {
            a.u_end[(size_t)(tr0 + 2 * pr) * nx + m] = ua;
            if (2 * pr + 1 < ntraj) a.u_end[(size_t)(tr0 + 2 * pr + 1) * nx + m] = ub;
        }
    }
    __syncthreads();
    if (save && a.norms) {
        dns_norms(Y, nx, ntraj, red);
        __syncthreads();
        if ((int)threadIdx.x < ntraj)
            a.norms[(size_t)(tr0 + threadIdx.x) * a.nsave + isave] = sqrt(a.L * red[threadIdx.x] * inx);
    }
    if (dst < 0) return;
    cpx<double>* F = fft_batch_r2<double, true>(Y, Z, lgnx, np, -1, tw, 0, twsh);
    const double* g = coef + 6 * nh;
    for (int i = threadIdx.x; i < np * nh; i += blockDim.x) {
        const int pr = i / nh, j = i - pr * nh;
        const cpx<double> P = F[(size_t)pr * nx + j];
        const cpx<double> Pm = conj(F[(size_t)pr * nx + ((nx - j) & (nx - 1))]);
        const cpx<double> sm = P + Pm, df = P - Pm;
        // W_a = (P + conj P_-j) / 2, W_b = (P - conj P_-j) / (2i); N = i g W
        const cpx<double> Wa = mk<double>(0.5 * sm.x, 0.5 * sm.y);
        const cpx<double> Wb = mk<double>(0.5 * df.y, -0.5 * df.x);
        spec(specs, nh, 2 * pr, dst)[j] = mk<double>(-g[j] * Wa.y, g[j] * Wa.x);
        if (2 * pr + 1 < ntraj) spec(specs, nh, 2 * pr + 1, dst)[j] = mk<double>(-g[j] * Wb.y, g[j] * Wb.x);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(DNS_THREADS) k_dns(DnsArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const DnsPlan pl = dns_plan(a.nx, a.nh, a.pairs);
    cpx<double>* tw = reinterpret_cast<cpx<double>*>(smem + pl.off_tw);
    double* coef = reinterpret_cast<double*>(smem + pl.off_coef);
    cpx<double>* fftb = reinterpret_cast<cpx<double>*>(smem + pl.off_fft);
    cpx<double>* specs = reinterpret_cast<cpx<double>*>(smem + pl.off_spec);
    double* red = reinterpret_cast<double*>(smem + pl.off_red);
    const int nx = a.nx, lgnx = a.lgnx, nh = a.nh;
    const int tr0 = blockIdx.x * 2 * a.pairs;
    const int ntraj = min(2 * a.pairs, a.batch - tr0);
    if (ntraj <= 0) return;
    const int np = (ntraj + 1) >> 1;
    const int twsh = LGNMAX - lgnx;

    // twiddles e^(2 pi i t / nx) at their swizzled slots of a compact table (see tw_swz)
    for (int t = threadIdx.x; t < nx; t += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)t / (double)nx, &s, &c);
        tw[tw_swz<double>(t)] = mk<double>(c, s);
    }
    dns_coefficients(coef, nh, a.L, a.dt);
    // analysis of u0: forward transform of the pairs, split, truncated to |j| <= Kx
    cpx<double>* A = fftb;
    cpx<double>* Bf = fftb + (size_t)a.pairs * nx;
    for (int i = threadIdx.x; i < np * nx; i += blockDim.x) {
        const int pr = i >> lgnx, m = i & (nx - 1);
        const double ua = a.u0[(size_t)(tr0 + 2 * pr) * nx + m];
        const double ub = (2 * pr + 1 < ntraj) ? a.u0[(size_t)(tr0 + 2 * pr + 1) * nx + m] : 0.0;
        A[i] = mk<double>(ua, ub);
    }
    __syncthreads();
    {
        cpx<double>* F = fft_batch_r2<double, true>(A, Bf, lgnx, np, -1, tw, 0, twsh);
        for (int i = threadIdx.x; i < np * nh; i += blockDim.x) {
            const int pr = i / nh, j = i - pr * nh;
            const cpx<double> P = F[(size_t)pr * nx + j];
            const cpx<double> Pm = conj(F[(size_t)pr * nx + ((nx - j) & (nx - 1))]);
            const cpx<double> sm = P + Pm, df = P - Pm;
            cpx<double> va = mk<double>(0.5 * sm.x, 0.5 * sm.y);
            cpx<double> vb = mk<double>(0.5 * df.y, -0.5 * df.x);
            if (a.symmetric) {
                va.x = 0.0;
                vb.x = 0.0;
            }
            spec(specs, nh, 2 * pr, SV)[j] = va;
            if (2 * pr + 1 < ntraj) spec(specs, nh, 2 * pr + 1, SV)[j] = vb;
        }
        __syncthreads();
    }

    const double* E = coef;
    const double* E2 = coef + nh;
    const double* Q = coef + 2 * nh;
    const double* f1 = coef + 3 * nh;
    const double* f2 = coef + 4 * nh;
    const double* f3 = coef + 5 * nh;
    const int nsp = ntraj * nh;
    for (long long n = 0; n < a.nsteps; ++n) {
        const long long isave = (n % a.save_every == 0) ? n / a.save_every : -1;
        dns_eval(a, tr0, ntraj, fftb, specs, tw, coef, red, SV, SNV, isave, false);
        for (int i = threadIdx.x; i < nsp; i += blockDim.x) {  // a = E2 v + Q Nv
            const int t = i / nh, j = i - t * nh;
            const cpx<double> v = spec(specs, nh, t, SV)[j], N = spec(specs, nh, t, SNV)[j];
            spec(specs, nh, t, SA)[j] = mk<double>(E2[j] * v.x + Q[j] * N.x, E2[j] * v.y + Q[j] * N.y);
        }
        __syncthreads();
        dns_eval(a, tr0, ntraj, fftb, specs, tw, coef, red, SA, SNA, -1, false);
        for (int i = threadIdx.x; i < nsp; i += blockDim.x) {  // b = E2 v + Q Na
            const int t = i / nh, j = i - t * nh;
            const cpx<double> v = spec(specs, nh, t, SV)[j], N = spec(specs, nh, t, SNA)[j];
            spec(specs, nh, t, SS)[j] = mk<double>(E2[j] * v.x + Q[j] * N.x, E2[j] * v.y + Q[j] * N.y);
        }
        __syncthreads();
        dns_eval(a, tr0, ntraj, fftb, specs, tw, coef, red, SS, SNB, -1, false);
        for (int i = threadIdx.x; i < nsp; i += blockDim.x) {  // c = E2 a + Q (2 Nb - Nv)
            const int t = i / nh, j = i - t * nh;
            const cpx<double> av = spec(specs, nh, t, SA)[j];
            const cpx<double> Nb = spec(specs, nh, t, SNB)[j], Nv = spec(specs, nh, t, SNV)[j];
            const cpx<double> d2 = mk<double>(2.0 * Nb.x - Nv.x, 2.0 * Nb.y - Nv.y);
            spec(specs, nh, t, SS)[j] = mk<double>(E2[j] * av.x + Q[j] * d2.x, E2[j] * av.y + Q[j] * d2.y);
        }
        __syncthreads();
        dns_eval(a, tr0, ntraj, fftb, specs, tw, coef, red, SS, SNC, -1, false);
        // v' = E v + f1 Nv + 2 f2 (Na + Nb) + f3 Nc; in the subspace the real parts are zeroed
        for (int i = threadIdx.x; i < nsp; i += blockDim.x) {
            const int t = i / nh, j = i - t * nh;
            const cpx<double> v = spec(specs, nh, t, SV)[j];
            const cpx<double> Nv = spec(specs, nh, t, SNV)[j], Na = spec(specs, nh, t, SNA)[j];
            const cpx<double> Nb = spec(specs, nh, t, SNB)[j], Nc = spec(specs, nh, t, SNC)[j];
            const double w2 = 2.0 * f2[j];
            cpx<double> vn = mk<double>(E[j] * v.x + f1[j] * Nv.x + w2 * (Na.x + Nb.x) + f3[j] * Nc.x,
                                        E[j] * v.y + f1[j] * Nv.y + w2 * (Na.y + Nb.y) + f3[j] * Nc.y);
            if (a.symmetric) vn.x = 0.0;
            spec(specs, nh, t, SV)[j] = vn;
        }
        __syncthreads();
    }
    const bool save_last = (a.nsteps % a.save_every == 0);
    if (save_last || a.u_end)
        dns_eval(a, tr0, ntraj, fftb, specs, tw, coef, red, SV, -1,
                 save_last ? a.nsteps / a.save_every : -1, true);
}

// Loop l of a segment cut: field at instants t_a + T_l n / Ns_l (n = 0..Ns_l - 1) by linear
// interpolation between the saved samples (sample i at time i * dts), written to the loop's
// ragged-packed slot [n][m] at out + off_l.
__global__ void k_dns_segment(const double* us, int nx, double dts, const int* a_idx, const double* T,
                              const int* ns, const long long* off, double* out) {
    const int l = blockIdx.x;
    const int nsl = ns[l], a0 = a_idx[l];
    const double Tl = T[l];
    for (int i = threadIdx.x; i < nsl * nx; i += blockDim.x) {
        const int n = i / nx, m = i - n * nx;
        const double x = (Tl * (double)n / (double)nsl) / dts;  // position in samples after a0
        int i0 = (int)floor(x);
        if (i0 < 0) i0 = 0;
        const double f = x - (double)i0;
        const double y0 = us[(size_t)(a0 + i0) * nx + m];
        const double y1 = us[(size_t)(a0 + i0 + 1) * nx + m];
        out[off[l] + i] = y0 + f * (y1 - y0);
    }
}

int dns_fail(int code, const std::string& msg) {
    ks_internal_set_error(msg.c_str());
    return code;
}

bool dns_is_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// A caller buffer as a device pointer: the buffer itself, or a temporary device copy (filled
// from the host when `in`), released and copied back by finish().
struct Staged {
    void* user = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    bool temp = false;
    bool out = false;
    int stage(void* p, size_t n, bool in, bool is_out, cudaStream_t s) {
        user = p;
        bytes = n;
        out = is_out;
        if (!p || n == 0) return KS_OK;
        if (dns_is_device(p)) {
            dev = p;
            return KS_OK;
        }
        if (cudaMalloc(&dev, n) != cudaSuccess) {
            cudaGetLastError();
            dev = nullptr;
            return dns_fail(KS_ERR_OOM, "device allocation for a host buffer failed");
        }
        temp = true;
        if (in && cudaMemcpyAsync(dev, p, n, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return dns_fail(KS_ERR_CUDA, "host to device copy failed");
        return KS_OK;
    }
    int finish(cudaStream_t s) {
        if (!temp) return KS_OK;
        int rc = KS_OK;
        if (out && cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            rc = dns_fail(KS_ERR_CUDA, "device to host copy failed");
        if (cudaStreamSynchronize(s) != cudaSuccess && rc == KS_OK)
            rc = dns_fail(KS_ERR_CUDA, "stream synchronisation failed");
        cudaFree(dev);
        temp = false;
        return rc;
    }
    ~Staged() {
        if (temp) cudaFree(dev);
    }
};

int ilog2i(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

extern "C" int ks_dns(double L, int nx, int batch, double dt, long long nsteps, int save_every,
                      int symmetric, const double* u0, double* u_saved, double* norms, double* u_end,
                      void* stream) {
    ks_internal_set_error("");
    if (!(L > 0.0) || !std::isfinite(L)) return dns_fail(KS_ERR_ARG, "L must be finite and > 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return dns_fail(KS_ERR_ARG, "dt must be finite and > 0");
    if (nx < 8 || nx > NMAX || (nx & (nx - 1))) return dns_fail(KS_ERR_ARG, "nx must be a power of two in [8, 1024]");
    if (batch < 1) return dns_fail(KS_ERR_ARG, "batch must be >= 1");
    if (nsteps < 0) return dns_fail(KS_ERR_ARG, "nsteps must be >= 0");
    if (save_every < 1) return dns_fail(KS_ERR_ARG, "save_every must be >= 1");
    if (!u0) return dns_fail(KS_ERR_ARG, "u0 is required");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return dns_fail(KS_ERR_CUDA, "no usable CUDA device");
    }
    cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    DnsArgs a{};
    a.L = L;
    a.dt = dt;
    a.nx = nx;
    a.lgnx = ilog2i(nx);
    a.kx = nx / 3;
    a.nh = a.kx + 1;
    a.batch = batch;
    a.save_every = save_every;
    a.symmetric = symmetric ? 1 : 0;
    a.nsteps = nsteps;
    a.nsave = nsteps / save_every + 1;
    // pairs per CTA: enough butterflies for the block (nx / 2 radix-2 butterflies per pair and
    // pass), within the shared memory of one CTA
    int pairs = std::max(1, std::min(DNS_PAIRS_MAX, (2 * DNS_THREADS) / nx));
    while (pairs > 1 && dns_plan(nx, a.nh, pairs).bytes > 200 * 1024) --pairs;
    pairs = std::min(pairs, (batch + 1) / 2);
    a.pairs = pairs;
    const DnsPlan pl = dns_plan(nx, a.nh, pairs);
    if (pl.bytes > 227 * 1024) return dns_fail(KS_ERR_ARG, "nx too large for the shared-memory plan");
    const size_t fb = (size_t)batch * nx * sizeof(double);
    Staged su0, ssv, snm, sue;
    int rc = su0.stage(const_cast<double*>(u0), fb, true, false, s);
    if (rc == KS_OK) rc = ssv.stage(u_saved, fb * (size_t)a.nsave, false, true, s);
    if (rc == KS_OK) rc = snm.stage(norms, (size_t)batch * a.nsave * sizeof(double), false, true, s);
    if (rc == KS_OK) rc = sue.stage(u_end, fb, false, true, s);
    if (rc != KS_OK) return rc;
    a.u0 = static_cast<const double*>(su0.dev);
    a.u_saved = static_cast<double*>(ssv.dev);
    a.norms = static_cast<double*>(snm.dev);
    a.u_end = static_cast<double*>(sue.dev);
    if (cudaFuncSetAttribute(k_dns, cudaFuncAttributeMaxDynamicSharedMemorySize, pl.bytes) != cudaSuccess) {
        cudaGetLastError();
        return dns_fail(KS_ERR_CUDA, "shared-memory attribute of the DNS kernel failed");
    }
    const int grid = (batch + 2 * pairs - 1) / (2 * pairs);
    k_dns<<<grid, DNS_THREADS, pl.bytes, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dns_fail(KS_ERR_CUDA, cudaGetErrorString(e));
    rc = su0.finish(s);
    int r2 = ssv.finish(s), r3 = snm.finish(s), r4 = sue.finish(s);
    if (rc == KS_OK) rc = r2;
    if (rc == KS_OK) rc = r3;
    if (rc == KS_OK) rc = r4;
    return rc;
}

extern "C" int ks_dns_segments(int nx, long long nsave, double dts, const double* us, int nloops,
                               const int* a_idx, const double* T, const int* ns, double* out,
                               void* stream) {
    ks_internal_set_error("");
    if (nx < 1 || nsave < 2 || !(dts > 0.0) || !std::isfinite(dts))
        return dns_fail(KS_ERR_ARG, "nx >= 1, nsave >= 2 and a finite dts > 0 are required");
    if (nloops < 0) return dns_fail(KS_ERR_ARG, "nloops must be >= 0");
    if (nloops == 0) return KS_OK;
    if (!us || !a_idx || !T || !ns || !out) return dns_fail(KS_ERR_ARG, "null pointer");
    // the per-loop tables are read here on the host
    if (dns_is_device(a_idx) || dns_is_device(T) || dns_is_device(ns))
        return dns_fail(KS_ERR_ARG, "a_idx, T and ns must be host arrays");
    std::vector<long long> off(nloops);
    long long tot = 0;
    for (int l = 0; l < nloops; ++l) {
        if (ns[l] < 1) return dns_fail(KS_ERR_ARG, "every Ns must be >= 1");
        if (!(T[l] > 0.0) || !std::isfinite(T[l])) return dns_fail(KS_ERR_ARG, "every T must be finite and > 0");
        // the last instant, a + T (Ns - 1) / Ns, and its right-hand sample must be saved
        const double last = T[l] * (double)(ns[l] - 1) / (double)ns[l] / dts;
        if (a_idx[l] < 0 || (double)a_idx[l] + std::floor(last) + 1.0 > (double)(nsave - 1))
            return dns_fail(KS_ERR_ARG, "a segment runs past the saved samples");
        off[l] = tot;
        tot += (long long)ns[l] * nx;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return dns_fail(KS_ERR_CUDA, "no usable CUDA device");
    }
    cudaGetLastError();
    cudaStream_t s = (cudaStream_t)stream;
    Staged sus, sout, sa, sT, sn, so;
    int rc = sus.stage(const_cast<double*>(us), (size_t)nsave * nx * sizeof(double), true, false, s);
    if (rc == KS_OK) rc = sout.stage(out, (size_t)tot * sizeof(double), false, true, s);
    // the per-loop tables always travel through a temporary device copy
    if (rc == KS_OK) rc = sa.stage(const_cast<int*>(a_idx), nloops * sizeof(int), true, false, s);
    if (rc == KS_OK) rc = sT.stage(const_cast<double*>(T), nloops * sizeof(double), true, false, s);
    if (rc == KS_OK) rc = sn.stage(const_cast<int*>(ns), nloops * sizeof(int), true, false, s);
    if (rc == KS_OK) rc = so.stage(off.data(), nloops * sizeof(long long), true, false, s);
    if (rc != KS_OK) return rc;
    k_dns_segment<<<nloops, 256, 0, s>>>(static_cast<const double*>(sus.dev), nx, dts,
                                         static_cast<const int*>(sa.dev), static_cast<const double*>(sT.dev),
                                         static_cast<const int*>(sn.dev), static_cast<const long long*>(so.dev),
                                         static_cast<double*>(sout.dev));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dns_fail(KS_ERR_CUDA, cudaGetErrorString(e));
    rc = sus.finish(s);
    int r2 = sout.finish(s);
    int r3 = sa.finish(s), r4 = sT.finish(s), r5 = sn.finish(s), r6 = so.finish(s);
    for (int r : {r2, r3, r4, r5, r6})
        if (rc == KS_OK) rc = r;
    return rc;
}
