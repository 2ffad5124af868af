// Host run of the per-CTA work items (ks_items.cuh compiled as sequential code with
// KS_HOST_EMULATION): one loop is analysed onto its band, takes `steps` tau-steps through the
// same four phases the per-phase launches run (ROW_NONLIN, COL_RESID, ROW_ADJ, COL_UPDATE), and
// is synthesised back to the grid.  Test infrastructure: the CPU tests compare its output with
// the oracle, so the items' index arithmetic and formulas are checked without a GPU.
//
// stdin:  L nx ns T dtau scheme steps, then ns * nx grid values u[n][m]
// stdout: sqrt(J) of the initial state, T after the steps, then ns * nx grid values
#include <cmath>
#include <cstdio>
#include <vector>

#define KS_HOST_EMULATION 1
#include "ks_items.cuh"

using namespace ks;

int main() {
    double L, T0, dtau;
    int nx, ns, scheme, steps;
    if (std::scanf("%lf %d %d %lf %lf %d %d", &L, &nx, &ns, &T0, &dtau, &scheme, &steps) != 7)
        return 2;
    std::vector<double> grid((size_t)ns * nx);
    for (auto& v : grid)
        if (std::scanf("%lf", &v) != 1) return 2;

    auto lg2 = [](int n) { int l = 0; while ((1 << l) < n) ++l; return l; };
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
    const int nkx = d.nkx, ks = ns / 3, nk = 2 * ks + 1;

    std::vector<int> v_ns{ns}, v_lg{lg2(ns)}, v_ks{ks}, v_colorder{0};
    std::vector<long long> v_zero{0};
    std::vector<cpx<double>> uh((size_t)nkx * nk), rh(uh.size()), gh(uh.size()), M((size_t)nkx * ns);
    std::vector<double> U((size_t)ns * nx), io(grid), T{T0, T0}, wT(2);
    wT[0] = wT[1] = 2.0 * 3.14159265358979323846 / T0;
    std::vector<double> Jpart(nkx), L2part(nkx), sqrtJ(1);
    std::vector<int> status{ST_RUNNING}, prec{0};
    std::vector<long long> nsteps{0};
    std::vector<cpx<double>> tw(NMAX);
    for (int t = 0; t < NMAX; ++t) {
        const double a = 2.0 * 3.14159265358979323846 * t / NMAX;
        tw[t] = mk<double>(std::cos(a), std::sin(a));
    }
    std::vector<double> qv(nkx), lin(nkx), cq(nkx), insv{1.0 / ns};
    for (int j = 0; j < nkx; ++j) {
        const double q = 2.0 * 3.14159265358979323846 * j / L;
        qv[j] = q;
        lin[j] = q * q - q * q * q * q;
        cq[j] = q * q * q * q * (q * q - 1.0) * (q * q - 1.0);
    }
    const int nr = ns < 8 ? ns : 8;
    std::vector<RowItem> rows;
    for (int n0 = 0; n0 < ns; n0 += nr) rows.push_back(RowItem{0, n0, nr, lg2(nr)});
    std::vector<double> smem_d(1 << 17);  // item scratch (8-byte aligned, 1 MiB)
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem_d.data());

    Bufs<double> p{};
    p.ns = v_ns.data();
    p.lgns = v_lg.data();
    p.ks = v_ks.data();
    p.boff = v_zero.data();
    p.moff = v_zero.data();
    p.goff = v_zero.data();
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
    p.steps = nsteps.data();
    p.sqrtJ = sqrtJ.data();
    p.tw = tw.data();
    p.qv = qv.data();
    p.lin = lin.data();
    p.cq = cq.data();
    p.insv = insv.data();
    p.rows = rows.data();
    p.colorder = v_colorder.data();
    p.myprec = 0;
    p.tol = 0.0;
    p.switch_tol = 0.0;
    const int nrow = (int)rows.size();

    // grid -> band, then the mixed values of the band (s-inverse)
    for (int it = 0; it < nrow; ++it) row_item<double, ROW_ANALYZE>(d, p, it, smem);
    for (int j = 0; j < nkx; ++j) col_item<double, COL_ANALYZE>(d, p, j, smem, 0);
    for (int j = 0; j < nkx; ++j) col_item<double, COL_SYNTH_U>(d, p, j, smem, 0);

    p.check_active = 1;
    double sqrtJ0 = -1.0;
    for (int s = 0; s < steps; ++s) {
        p.par = s & 1;
        for (int it = 0; it < nrow; ++it) row_item<double, ROW_NONLIN>(d, p, it, smem);
        for (int j = 0; j < nkx; ++j) col_item<double, COL_RESID>(d, p, j, smem, p.par);
        for (int it = 0; it < nrow; ++it) row_item<double, ROW_ADJ>(d, p, it, smem);
        for (int j = 0; j < nkx; ++j) col_item<double, COL_UPDATE>(d, p, j, smem, p.par);
        if (s == 0) sqrtJ0 = sqrtJ[0];
    }

    // band -> grid
    p.check_active = 0;
    for (int j = 0; j < nkx; ++j) col_item<double, COL_SYNTH_U>(d, p, j, smem, 0);
    for (int it = 0; it < nrow; ++it) row_item<double, ROW_SYNTH>(d, p, it, smem);

    std::printf("%.17g %.17g\n", sqrtJ0, T[steps & 1]);
    for (size_t i = 0; i < io.size(); ++i) std::printf("%.17g\n", io[i]);
    return 0;
}
