// Host run of the per-CTA work items (ks_items.cuh compiled as sequential code with
// KS_HOST_EMULATION).  One loop is analysed onto its band (in double, as the library always
// does), rounded to the working precision, and then either
//   mode 0: takes `steps` tau-steps through the four phases the per-phase launches run
//           (ROW_NONLIN, COL_RESID, ROW_ADJ, COL_UPDATE) and is synthesised back to the grid, or
//   mode 1: has its residual and adjoint gradient evaluated (COL_SYNTH_U, ROW_NONLIN, COL_RESID,
//           ROW_ADJ, COL_GRAD) and G synthesised to the grid, with J and dJ/dT from the column
//           partials summed in the fixed order of the finalising kernel, or
//   mode 2: the same residual pass only, with r synthesised to the grid (COL_SYNTH_R).
// Test infrastructure: the CPU tests compare its output with the oracle, so the items' index
// arithmetic and formulas are checked without a GPU.
//
// stdin:  L nx ns T dtau scheme steps mode prec(64|32) xi(0|1), then ns * nx values u[n][m]
// stdout: mode 0: sqrt(J) of the initial state, T after the steps, then the grid u
//         mode 1: J, dJ/dT, then the grid G; mode 2: J, dJ/dT, then the grid r
#include <cmath>
#include <cstdio>
#include <vector>

#define KS_HOST_EMULATION 1
#include "ks_items.cuh"

using namespace ks;

namespace {

const double kPi = 3.14159265358979323846;

int lg2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Host copies of every buffer of one precision, and the Bufs that point into them.
template <typename R>
struct HostLoop {
    std::vector<int> ns, lgns, ks, colorder{0};
    std::vector<long long> zero{0}, steps{0};
    std::vector<cpx<R>> uh, rh, gh, M, tw;
    std::vector<R> U, io, qv, lin, cq, insv;
    std::vector<double> T, wT, sqrtJ{0.0};
    std::vector<typename PartT<R>::type> Jpart, L2part;
    std::vector<int> status{ST_RUNNING}, prec;
    std::vector<RowItem> rows;
    Bufs<R> p{};

    HostLoop(const Dims& d, int n, double T0, int xi) {
        const int nkx = d.nkx, k3 = n / 3, nk = 2 * k3 + 1;
        ns = {n};
        lgns = {lg2(n)};
        ks = {k3};
        uh.assign((size_t)nkx * nk, mk<R>(0, 0));
        rh = gh = uh;
        M.assign((size_t)nkx * n, mk<R>(0, 0));
        U.assign((size_t)n * d.nx, 0);
        io = U;
        T = {T0, T0};
        wT = {2.0 * kPi / T0, 2.0 * kPi / T0};
        Jpart.resize(nkx);
        L2part.resize(nkx);
        prec = {sizeof(R) == 8 ? 0 : 1};
        tw.resize(NMAX);
        for (int t = 0; t < NMAX; ++t) {
            const double a = 2.0 * kPi * t / NMAX;
            tw[t] = mk<R>((R)std::cos(a), (R)std::sin(a));
        }
        for (int j = 0; j < nkx; ++j) {
            const double q = 2.0 * kPi * j / d.L;
            qv.push_back((R)q);
            lin.push_back((R)(q * q - q * q * q * q));
            cq.push_back((R)(q * q * q * q * (q * q - 1.0) * (q * q - 1.0)));
        }
        insv = {(R)(1.0 / n)};
        const int nr = n < 8 ? n : 8;
        for (int n0 = 0; n0 < n; n0 += nr) rows.push_back(RowItem{0, n0, nr, lg2(nr)});
        p.ns = ns.data();
        p.lgns = lgns.data();
        p.ks = ks.data();
        p.boff = p.moff = p.goff = zero.data();
        p.uh = uh.data();
        p.rh = rh.data();
        p.gh = gh.data();
        p.M = M.data();
        p.U = U.data();
        p.io = io.data();
        p.T = T.data();
        p.wT = wT.data();
        p.Jpart = Jpart.data();
        p.L2part = L2part.data();
        p.status = status.data();
        p.prec = prec.data();
        p.steps = steps.data();
        p.sqrtJ = sqrtJ.data();
        p.tw = tw.data();
        p.qv = qv.data();
        p.lin = lin.data();
        p.cq = cq.data();
        p.insv = insv.data();
        p.rows = rows.data();
        p.colorder = colorder.data();
        p.myprec = prec[0];
        p.xi = xi;
    }
};

template <typename R>
int run(const Dims& d, int ns, double T0, int xi, int steps, int mode,
        const std::vector<cpx<double>>& band) {
    HostLoop<R> h(d, ns, T0, xi);
    Bufs<R>& p = h.p;
    for (size_t i = 0; i < band.size(); ++i) h.uh[i] = mk<R>((R)band[i].x, (R)band[i].y);
    std::vector<double> smem_d(1 << 17);  // item scratch (1 MiB)
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem_d.data());
    const int nrow = (int)h.rows.size(), nkx = d.nkx;

    for (int j = 0; j < nkx; ++j) col_item<R, COL_SYNTH_U>(d, p, j, smem, 0);
    if (mode == 0) {
        p.check_active = 1;
        double sqrtJ0 = -1.0;
        for (int s = 0; s < steps; ++s) {
            p.par = s & 1;
            for (int it = 0; it < nrow; ++it) row_item<R, ROW_NONLIN>(d, p, it, smem);
            for (int j = 0; j < nkx; ++j) col_item<R, COL_RESID>(d, p, j, smem, p.par);
            for (int it = 0; it < nrow; ++it) row_item<R, ROW_ADJ>(d, p, it, smem);
            for (int j = 0; j < nkx; ++j) col_item<R, COL_UPDATE>(d, p, j, smem, p.par);
            if (s == 0) sqrtJ0 = h.sqrtJ[0];
        }
        p.check_active = 0;
        for (int j = 0; j < nkx; ++j) col_item<R, COL_SYNTH_U>(d, p, j, smem, 0);
        for (int it = 0; it < nrow; ++it) row_item<R, ROW_SYNTH>(d, p, it, smem);
        std::printf("%.17g %.17g\n", sqrtJ0, h.T[steps & 1]);
    } else {
        for (int it = 0; it < nrow; ++it) row_item<R, ROW_NONLIN>(d, p, it, smem);
        for (int j = 0; j < nkx; ++j) col_item<R, COL_RESID>(d, p, j, smem, 0);
        if (mode == 1) {
            for (int it = 0; it < nrow; ++it) row_item<R, ROW_ADJ>(d, p, it, smem);
            for (int j = 0; j < nkx; ++j) col_item<R, COL_GRAD>(d, p, j, smem, 0);
        }
        // J and dJ/dT = 2 L^dag_2 from the partials, in column order as the finalising kernel
        double sj = 0.0, sl = 0.0;
        for (int c = 0; c < nkx; ++c) {
            sj += widen(h.Jpart[c]);
            sl += widen(h.L2part[c]);
        }
        const double J = d.L * sj, dJdT = 2.0 * d.L * 2.0 * kPi * sl / (T0 * T0);
        if (mode == 1)
            for (int j = 0; j < nkx; ++j) col_item<R, COL_SYNTH_G>(d, p, j, smem, 0);
        else
            for (int j = 0; j < nkx; ++j) col_item<R, COL_SYNTH_R>(d, p, j, smem, 0);
        for (int it = 0; it < nrow; ++it) row_item<R, ROW_SYNTH>(d, p, it, smem);
        std::printf("%.17g %.17g\n", J, dJdT);
    }
    for (size_t i = 0; i < h.io.size(); ++i) std::printf("%.17g\n", (double)h.io[i]);
    return 0;
}

}  // namespace

int main() {
    double L, T0, dtau;
    int nx, ns, scheme, steps, mode, precision, xi;
    if (std::scanf("%lf %d %d %lf %lf %d %d %d %d %d", &L, &nx, &ns, &T0, &dtau, &scheme, &steps,
                   &mode, &precision, &xi) != 10)
        return 2;
    Dims d{};
    d.B = 1;
    d.nx = nx;
    d.lgnx = lg2(nx);
    d.kx = nx / 3;
    d.nkx = d.kx + 1;
    d.L = L;
    d.dtau = dtau;
    d.scheme = scheme;
    d.hx = 0.5 / nx;

    // analysis onto the band, always in double
    HostLoop<double> a(d, ns, T0, xi);
    for (auto& v : a.io)
        if (std::scanf("%lf", &v) != 1) return 2;
    std::vector<double> smem_d(1 << 17);
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem_d.data());
    for (int it = 0; it < (int)a.rows.size(); ++it) row_item<double, ROW_ANALYZE>(d, a.p, it, smem);
    for (int j = 0; j < d.nkx; ++j) col_item<double, COL_ANALYZE>(d, a.p, j, smem, 0);

    if (precision == 32) return run<float>(d, ns, T0, xi, steps, mode, a.uh);
    return run<double>(d, ns, T0, xi, steps, mode, a.uh);
}
