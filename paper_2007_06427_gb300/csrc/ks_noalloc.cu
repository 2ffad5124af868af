// ks_noalloc.cu - residual of one loop with no device allocation.
//
// Some callers cannot allocate device memory at the point where they need a residual: code
// running inside a pre-sized memory pool or arena that owns all of the device memory, plugins
// of a host application that forbids allocation after start-up, or real-time loops where a
// cudaMalloc (an implicit device synchronisation and a possible failure) is not acceptable.
// For them ks_residual_noalloc computes the same result as ks_residual for one double-precision
// loop without a handle: every intermediate lives in one file-scope device array of fixed size
// (KS_NOALLOC_BYTES), reserved when the library is loaded.
//
// The kernels are the same per-CTA items as the handle-based path (ks_items.cuh); only the
// place of the scratch differs.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "ks_items.cuh"
#include "ks_loop.h"

using namespace ks;

namespace {

constexpr int NA_NXMAX = 256;
constexpr int NA_NSMAX = 256;
constexpr int NA_NKX = NA_NXMAX / 3 + 1;
constexpr int NA_NK = 2 * (NA_NSMAX / 3) + 1;
constexpr int NA_ROWS = 2;  // rows per tile
constexpr int NA_ITEMS = NA_NSMAX / NA_ROWS;
constexpr int NA_THREADS = 128;

constexpr size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

// byte offsets of the pieces inside the scratch array (sized for the maxima above)
constexpr size_t O_TW = 0;
constexpr size_t O_QV = O_TW + al(sizeof(cpx<double>) * NMAX);
constexpr size_t O_LIN = O_QV + al(sizeof(double) * NA_NKX);
constexpr size_t O_CQ = O_LIN + al(sizeof(double) * NA_NKX);
constexpr size_t O_SCAL = O_CQ + al(sizeof(double) * NA_NKX);  // insv, T[2], wT[2], J, dJdT, sqrtJ
constexpr size_t O_INT = O_SCAL + al(sizeof(double) * 16);    // ns, lgns, ks, colorder, status, prec
constexpr size_t O_OFF = O_INT + al(sizeof(int) * 16);        // boff, moff, goff, steps
constexpr size_t O_ROWS = O_OFF + al(sizeof(long long) * 8);
constexpr size_t O_JP = O_ROWS + al(sizeof(RowItem) * NA_ITEMS);
constexpr size_t O_LP = O_JP + al(sizeof(double) * NA_NKX);
constexpr size_t O_UH = O_LP + al(sizeof(double) * NA_NKX);
constexpr size_t O_RH = O_UH + al(sizeof(cpx<double>) * NA_NKX * NA_NK);
constexpr size_t O_M = O_RH + al(sizeof(cpx<double>) * NA_NKX * NA_NK);
constexpr size_t O_U = O_M + al(sizeof(cpx<double>) * NA_NKX * NA_NSMAX);
constexpr size_t O_END = O_U + al(sizeof(double) * NA_NSMAX * NA_NXMAX);

}  // namespace

// KS_NOALLOC_BYTES: size of the scratch array (about 1.4 MB).  Every GPU that loads the
// library holds it until the process exits.
#define KS_NOALLOC_BYTES O_END

static __device__ __align__(256) unsigned char g_ks_noalloc_scratch[KS_NOALLOC_BYTES];

namespace {

// per-call tables: sizes of the single loop, wavenumber tables, row items, T
__global__ void k_na_prep(unsigned char* base, double L, int nx, int ns, double T) {
    const int nkx = nx / 3 + 1;
    double* qv = reinterpret_cast<double*>(base + O_QV);
    double* lin = reinterpret_cast<double*>(base + O_LIN);
    double* cq = reinterpret_cast<double*>(base + O_CQ);
    double* sc = reinterpret_cast<double*>(base + O_SCAL);
    int* iv = reinterpret_cast<int*>(base + O_INT);
    long long* off = reinterpret_cast<long long*>(base + O_OFF);
    RowItem* rows = reinterpret_cast<RowItem*>(base + O_ROWS);
    for (int j = threadIdx.x; j < nkx; j += blockDim.x) {
        const double q = 2.0 * 3.14159265358979323846 * (double)j / L;
        qv[j] = q;
        lin[j] = q * q - q * q * q * q;
        cq[j] = q * q * q * q * (q * q - 1.0) * (q * q - 1.0);
    }
    for (int i = threadIdx.x; i < ns / NA_ROWS; i += blockDim.x)
        rows[i] = RowItem{0, i * NA_ROWS, NA_ROWS, 1};
    if (threadIdx.x == 0) {
        int lg = 0;
        while ((1 << lg) < ns) ++lg;
        sc[0] = 1.0 / (double)ns;                      // insv
        sc[1] = T;                                     // T[0]
        sc[2] = T;                                     // T[1]
        sc[3] = 2.0 * 3.14159265358979323846 / T;      // wT[0]
        sc[4] = sc[3];                                 // wT[1]
        sc[5] = sc[6] = sc[7] = 0.0;                   // J, dJdT, sqrtJ
        iv[0] = ns;
        iv[1] = lg;
        iv[2] = ns / 3;
        iv[3] = 0;                                     // colorder
        iv[4] = 0;                                     // status
        iv[5] = 0;                                     // prec (double)
        off[0] = off[1] = off[2] = 0;                  // band / mixed / grid offsets
        off[3] = 0;                                    // steps
    }
}

template <int MODE>
__global__ void __launch_bounds__(NA_THREADS) k_na_rows(Dims d, Bufs<double> p, int nitems) {
    extern __shared__ __align__(16) unsigned char smem[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) row_item<double, MODE>(d, p, it, smem);
}

template <int MODE>
__global__ void __launch_bounds__(NA_THREADS) k_na_cols(Dims d, Bufs<double> p, int nitems) {
    extern __shared__ __align__(16) unsigned char smem[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) col_item<double, MODE>(d, p, it, smem, 0);
}

__global__ void k_na_finalize(int nkx, double L, const double* Jpart, double* J) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int c = 0; c < nkx; ++c) s += Jpart[c];
        *J = L * s;
    }
}

// host-side twiddles exp(2 pi i t / NMAX), octant symmetric (held in static host storage)
void na_twiddles(cpx<double>* tw) {
    const int N = NMAX;
    const double two_pi = 6.283185307179586476925286766559;
    static double c[NMAX / 4 + 1], s[NMAX / 4 + 1];
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
        const double a = c[r], b = s[r];
        double re, im;
        switch (qd) {
            case 0: re = a; im = b; break;
            case 1: re = -b; im = a; break;
            case 2: re = -a; im = -b; break;
            default: re = b; im = -a; break;
        }
        tw[t].x = re;
        tw[t].y = im;
    }
}

constexpr int NA_MAXDEV = 64;
std::mutex g_na_mutex;
unsigned char* g_na_base[NA_MAXDEV] = {nullptr};
// the context the set-up of each device was done in: a device reset or a context torn down and
// created again reloads the module, which leaves the array without its twiddle table (and may
// move it), so a new context id triggers the set-up again
unsigned long long g_na_ctx[NA_MAXDEV] = {0};

}  // namespace

// message for ks_last_error() (defined with the other entry points)
void ks_internal_set_error(const char* msg);

namespace {

int na_fail(int code, const char* msg) {
    ks_internal_set_error(msg);
    return code;
}

// Once per device, with that device current: the device address of the scratch array (the
// host-side symbol is only a stand-in), the twiddle table copied into it, and the shared
// memory limits of the kernels.
// Id of the current context (the driver's cuCtxGetCurrent / cuCtxGetId, reached through the
// runtime's entry-point query so that the library needs no link against the driver library).
int na_context_id(unsigned long long* id) {
    typedef int (*get_current_t)(void**);
    typedef int (*get_id_t)(void*, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            cudaGetLastError();
            return na_fail(KS_ERR_CUDA, "the driver's context queries are not available");
        }
        get_current = reinterpret_cast<get_current_t>(f1);
        get_id = reinterpret_cast<get_id_t>(f2);
    }
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, id) != 0)
        return na_fail(KS_ERR_CUDA, "no current CUDA context");
    return KS_OK;
}

int na_setup(int dev, unsigned char** base) {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    unsigned long long ctx = 0;
    int rc = na_context_id(&ctx);
    if (rc != KS_OK) return rc;
    if (g_na_base[dev] && g_na_ctx[dev] == ctx) {
        *base = g_na_base[dev];
        return KS_OK;
    }
    g_na_base[dev] = nullptr;
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_ks_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return na_fail(KS_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
    }
    static cpx<double> tw[NMAX];
    na_twiddles(tw);
    e = cudaMemcpy(static_cast<unsigned char*>(ptr) + O_TW, tw, sizeof(tw), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return na_fail(KS_ERR_CUDA, "twiddle upload failed");
    const int rs = (int)(2 * NA_ROWS * NA_NXMAX * sizeof(cpx<double>));
    const int cs = (int)(2 * NA_NSMAX * sizeof(cpx<double>) + COL_RED_DOUBLES * sizeof(double));
    if (cudaFuncSetAttribute(k_na_rows<ROW_ANALYZE>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs) ||
        cudaFuncSetAttribute(k_na_rows<ROW_NONLIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs) ||
        cudaFuncSetAttribute(k_na_rows<ROW_SYNTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs) ||
        cudaFuncSetAttribute(k_na_cols<COL_ANALYZE>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs) ||
        cudaFuncSetAttribute(k_na_cols<COL_SYNTH_U>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs) ||
        cudaFuncSetAttribute(k_na_cols<COL_SYNTH_R>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs) ||
        cudaFuncSetAttribute(k_na_cols<COL_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) {
        cudaGetLastError();
        return na_fail(KS_ERR_CUDA, "kernel attribute setup failed");
    }
    g_na_base[dev] = static_cast<unsigned char*>(ptr);
    g_na_ctx[dev] = ctx;
    *base = g_na_base[dev];
    return KS_OK;
}

// device (or managed) memory of device dev
bool na_is_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

static_assert(KS_NOALLOC_BYTES <= 2 * 1024 * 1024, "the no-allocation scratch must stay modest");

extern "C" int ks_residual_noalloc(double L, int nx, int ns, const double* u, double T, double* r,
                                   double* J, void* stream) {
    ks_internal_set_error("");
    cudaGetLastError();  // an error left by an unrelated earlier launch is not this call's
    if (!(L > 0.0) || !std::isfinite(L)) return na_fail(KS_ERR_ARG, "L must be > 0");
    if (!(T > 0.0) || !std::isfinite(T)) return na_fail(KS_ERR_ARG, "T must be finite and > 0");
    if (nx < 8 || nx > NA_NXMAX || (nx & (nx - 1)))
        return na_fail(KS_ERR_ARG, "nx must be a power of two in [8, 256] for the no-allocation call");
    if (ns < 8 || ns > NA_NSMAX || (ns & (ns - 1)))
        return na_fail(KS_ERR_ARG, "ns must be a power of two in [8, 256] for the no-allocation call");
    if (!u || !J) return na_fail(KS_ERR_ARG, "u and J are required");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAXDEV) {
        cudaGetLastError();
        return na_fail(KS_ERR_CUDA, "no usable CUDA device");
    }
    if (!na_is_device(u, dev) || !na_is_device(J, dev) || (r && !na_is_device(r, dev)))
        return na_fail(KS_ERR_ARG, "the no-allocation call takes device pointers of the current device only");
    unsigned char* base = nullptr;
    int rc = na_setup(dev, &base);
    if (rc != KS_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    Dims d{};
    d.B = 1;
    d.nx = nx;
    int lgnx = 0;
    while ((1 << lgnx) < nx) ++lgnx;
    d.lgnx = lgnx;
    d.kx = nx / 3;
    d.nkx = d.kx + 1;
    d.L = L;
    d.dtau = 0.0;
    d.scheme = 1;
    d.hx = 0.5 / (double)nx;

    Bufs<double> p{};
    int* iv = reinterpret_cast<int*>(base + O_INT);
    long long* off = reinterpret_cast<long long*>(base + O_OFF);
    double* sc = reinterpret_cast<double*>(base + O_SCAL);
    p.ns = iv + 0;
    p.lgns = iv + 1;
    p.ks = iv + 2;
    p.colorder = iv + 3;
    p.status = iv + 4;
    p.prec = iv + 5;
    p.boff = off + 0;
    p.moff = off + 1;
    p.goff = off + 2;
    p.steps = off + 3;
    p.uh = reinterpret_cast<cpx<double>*>(base + O_UH);
    p.rh = reinterpret_cast<cpx<double>*>(base + O_RH);
    p.gh = nullptr;
    p.M = reinterpret_cast<cpx<double>*>(base + O_M);
    p.U = reinterpret_cast<double*>(base + O_U);
    p.T = sc + 1;
    p.wT = sc + 3;
    p.sqrtJ = sc + 7;
    p.Jpart = reinterpret_cast<double*>(base + O_JP);
    p.L2part = reinterpret_cast<double*>(base + O_LP);
    p.tw = reinterpret_cast<const cpx<double>*>(base + O_TW);
    p.qv = reinterpret_cast<const double*>(base + O_QV);
    p.lin = reinterpret_cast<const double*>(base + O_LIN);
    p.cq = reinterpret_cast<const double*>(base + O_CQ);
    p.insv = sc + 0;
    p.rows = reinterpret_cast<const RowItem*>(base + O_ROWS);
    p.myprec = 0;
    p.par = 0;
    p.check_active = 0;

    const int nrow = ns / NA_ROWS;
    const int ncol = d.nkx;
    const size_t rs = 2 * (size_t)NA_ROWS * nx * sizeof(cpx<double>);
    const size_t cs = 2 * (size_t)ns * sizeof(cpx<double>) + COL_RED_DOUBLES * sizeof(double);
    k_na_prep<<<1, NA_THREADS, 0, s>>>(base, L, nx, ns, T);
    // project u onto the band (a4 applied to the input), then a1-a6 and the synthesis of r
    p.io = const_cast<double*>(u);
    k_na_rows<ROW_ANALYZE><<<nrow, NA_THREADS, rs, s>>>(d, p, nrow);
    k_na_cols<COL_ANALYZE><<<ncol, NA_THREADS, cs, s>>>(d, p, ncol);
    k_na_cols<COL_SYNTH_U><<<ncol, NA_THREADS, cs, s>>>(d, p, ncol);
    k_na_rows<ROW_NONLIN><<<nrow, NA_THREADS, rs, s>>>(d, p, nrow);
    k_na_cols<COL_RESID><<<ncol, NA_THREADS, cs, s>>>(d, p, ncol);
    k_na_finalize<<<1, 32, 0, s>>>(ncol, L, reinterpret_cast<const double*>(base + O_JP), J);
    if (r) {
        p.io = r;
        k_na_cols<COL_SYNTH_R><<<ncol, NA_THREADS, cs, s>>>(d, p, ncol);
        k_na_rows<ROW_SYNTH><<<nrow, NA_THREADS, rs, s>>>(d, p, nrow);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(KS_ERR_CUDA, cudaGetErrorString(e));
    return KS_OK;
}
