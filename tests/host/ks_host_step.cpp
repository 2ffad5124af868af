// Host run of the per-CTA work items (ks_items.cuh compiled as sequential code with
// KS_HOST_EMULATION) over a ragged batch of loops, laid out as the library lays them out (band,
// mixed and grid offsets per loop, columns longest loop first, row tiles per loop).  The batch is
// analysed onto its bands (in double, as the library always does), rounded to the working
// precision, and then either
//   mode 0: takes `steps` tau-steps through the four phases the per-phase launches run
//           (ROW_NONLIN, COL_RESID, ROW_ADJ, COL_UPDATE) and is synthesised back to the grid, or
//   mode 1: has its residual and adjoint gradient evaluated (COL_SYNTH_U, ROW_NONLIN, COL_RESID,
//           ROW_ADJ, COL_GRAD) and G synthesised to the grid, with J and dJ/dT from the column
//           partials summed in the fixed order of the finalising kernel, or
//   mode 2: the same residual pass only, with r synthesised to the grid (COL_SYNTH_R).
// Test infrastructure: the CPU tests compare its output with the oracle, so the items' index
// arithmetic and formulas are checked without a GPU.
//
// stdin:  L nx B dtau scheme steps mode prec(64|32) xi(0|1) tol switch_tol, then B pairs "Ns_b T_b", then
//         the grid values of every loop, loop after loop, each u[n][m]
// stdout: B lines "a_b c_b s_b n_b" (mode 0: sqrt(J) of the initial state, T after the steps,
//         the loop's status and steps taken; modes 1, 2: J, dJ/dT, 0, 0), then the grid values
//         (u, G or r) of every loop in order
#include <algorithm>
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

// Host copies of every buffer of one precision for the whole batch, and the Bufs into them.
template <typename R>
struct HostBatch {
    std::vector<int> ns, lgns, ks, colorder, status, prec;
    std::vector<long long> boff, moff, goff, steps;
    std::vector<cpx<R>> uh, rh, gh, M, tw;
    std::vector<R> U, io, qv, lin, cq, insv;
    std::vector<double> T, wT, sqrtJ;
    std::vector<typename PartT<R>::type> Jpart, L2part;
    std::vector<RowItem> rows;
    Bufs<R> p{};

    HostBatch(const Dims& d, const std::vector<int>& nsv, const std::vector<double>& T0, int xi) {
        const int B = d.B, nkx = d.nkx;
        long long bo = 0, mo = 0, go = 0;
        for (int b = 0; b < B; ++b) {
            const int n = nsv[b];
            ns.push_back(n);
            lgns.push_back(lg2(n));
            ks.push_back(n / 3);
            boff.push_back(bo);
            moff.push_back(mo);
            goff.push_back(go);
            bo += (long long)nkx * (2 * (n / 3) + 1);
            mo += (long long)nkx * n;
            go += (long long)n * d.nx;
            insv.push_back((R)(1.0 / n));
        }
        uh.assign(bo, mk<R>(0, 0));
        rh = gh = uh;
        M.assign(mo, mk<R>(0, 0));
        U.assign(go, 0);
        io = U;
        T.resize(2 * B);
        wT.resize(2 * B);
        for (int b = 0; b < B; ++b) {
            T[b] = T[B + b] = T0[b];
            wT[b] = wT[B + b] = 2.0 * kPi / T0[b];
        }
        Jpart.resize((size_t)B * nkx);
        L2part.resize((size_t)B * nkx);
        status.assign(B, ST_RUNNING);
        prec.assign(B, sizeof(R) == 8 ? 0 : 1);
        steps.assign(B, 0);
        sqrtJ.assign(B, 0.0);
        // columns of the longest loops first (the library's order); rows in tiles of <= 8
        for (int b = 0; b < B; ++b) colorder.push_back(b);
        std::stable_sort(colorder.begin(), colorder.end(),
                         [&](int a, int c) { return ns[a] > ns[c]; });
        for (int b = 0; b < B; ++b) {
            const int nr = std::min(ns[b], 8);
            for (int n0 = 0; n0 < ns[b]; n0 += nr) rows.push_back(RowItem{b, n0, nr, lg2(nr)});
        }
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
        point();
        p.xi = xi;
    }

    void point() {
        p.ns = ns.data();
        p.lgns = lgns.data();
        p.ks = ks.data();
        p.boff = boff.data();
        p.moff = moff.data();
        p.goff = goff.data();
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
    }
};

std::vector<double> g_smem(1 << 17);  // item scratch (1 MiB)

template <typename R>
void rows_pass(const Dims& d, HostBatch<R>& h, int mode) {
    unsigned char* smem = reinterpret_cast<unsigned char*>(g_smem.data());
    for (int it = 0; it < (int)h.rows.size(); ++it) {
        switch (mode) {
            case ROW_ANALYZE: row_item<R, ROW_ANALYZE>(d, h.p, it, smem); break;
            case ROW_NONLIN: row_item<R, ROW_NONLIN>(d, h.p, it, smem); break;
            case ROW_ADJ: row_item<R, ROW_ADJ>(d, h.p, it, smem); break;
            default: row_item<R, ROW_SYNTH>(d, h.p, it, smem); break;
        }
    }
}

template <typename R, int MODE>
void cols_pass(const Dims& d, HostBatch<R>& h, int par) {
    unsigned char* smem = reinterpret_cast<unsigned char*>(g_smem.data());
    for (int it = 0; it < col_item_count(d, h.p.xi, MODE); ++it) col_item<R, MODE>(d, h.p, it, smem, par);
}

template <typename R>
int run(const Dims& d, const std::vector<int>& nsv, const std::vector<double>& T0, int xi,
        int steps, int mode, double tol, double switch_tol,
        const std::vector<cpx<double>>& band) {
    HostBatch<R> h(d, nsv, T0, xi);
    Bufs<R>& p = h.p;
    p.tol = tol;
    p.switch_tol = switch_tol;
    for (size_t i = 0; i < band.size(); ++i) h.uh[i] = mk<R>((R)band[i].x, (R)band[i].y);
    const int B = d.B, nkx = d.nkx;
    std::vector<double> a(B), c(B);

    cols_pass<R, COL_SYNTH_U>(d, h, 0);
    if (mode == 0) {
        p.check_active = 1;
        p.step_scalars = 1;  // each loop's step scalars after the ROW_ADJ items, as in the launches
        for (int s = 0; s < steps; ++s) {
            p.par = s & 1;
            rows_pass<R>(d, h, ROW_NONLIN);
            cols_pass<R, COL_RESID>(d, h, p.par);
            rows_pass<R>(d, h, ROW_ADJ);
            loops_scalars(d, p, p.par, 0, 1);  // after the ROW_ADJ items, as the launches do
            cols_pass<R, COL_UPDATE>(d, h, p.par);
            if (s == 0) a = h.sqrtJ;
        }
        p.check_active = 0;
        p.step_scalars = 0;
        for (int b = 0; b < B; ++b) c[b] = h.T[(size_t)(steps & 1) * B + b];
        cols_pass<R, COL_SYNTH_U>(d, h, 0);
    } else {
        rows_pass<R>(d, h, ROW_NONLIN);
        cols_pass<R, COL_RESID>(d, h, 0);
        if (mode == 1) {
            rows_pass<R>(d, h, ROW_ADJ);
            cols_pass<R, COL_GRAD>(d, h, 0);
        }
        // J and dJ/dT = 2 L^dag_2 from the partials, in column order as the finalising kernel
        for (int b = 0; b < B; ++b) {
            double sj = 0.0, sl = 0.0;
            for (int k = 0; k < nkx; ++k) {
                sj += widen(h.Jpart[(size_t)b * nkx + k]);
                sl += widen(h.L2part[(size_t)b * nkx + k]);
            }
            a[b] = d.L * sj;
            c[b] = 2.0 * d.L * 2.0 * kPi * sl / (T0[b] * T0[b]);
        }
        if (mode == 1) cols_pass<R, COL_SYNTH_G>(d, h, 0);
        else cols_pass<R, COL_SYNTH_R>(d, h, 0);
    }
    rows_pass<R>(d, h, ROW_SYNTH);
    for (int b = 0; b < B; ++b)
        std::printf("%.17g %.17g %d %lld\n", a[b], c[b], mode == 0 ? h.status[b] : 0,
                    mode == 0 ? h.steps[b] : 0LL);
    for (size_t i = 0; i < h.io.size(); ++i) std::printf("%.17g\n", (double)h.io[i]);
    return 0;
}

}  // namespace

int main() {
    double L, dtau;
    double tol, switch_tol;
    int nx, B, scheme, steps, mode, precision, xi;
    if (std::scanf("%lf %d %d %lf %d %d %d %d %d %lf %lf", &L, &nx, &B, &dtau, &scheme, &steps,
                   &mode, &precision, &xi, &tol, &switch_tol) != 11 || B < 1)
        return 2;
    std::vector<int> nsv(B);
    std::vector<double> T0(B);
    for (int b = 0; b < B; ++b)
        if (std::scanf("%d %lf", &nsv[b], &T0[b]) != 2) return 2;
    Dims d{};
    d.B = B;
    d.nx = nx;
    d.lgnx = lg2(nx);
    d.kx = nx / 3;
    d.nkx = d.kx + 1;
    d.L = L;
    d.dtau = dtau;
    d.scheme = scheme;
    d.hx = 0.5 / nx;

    // analysis onto the bands, always in double
    HostBatch<double> an(d, nsv, T0, xi);
    for (auto& v : an.io)
        if (std::scanf("%lf", &v) != 1) return 2;
    rows_pass<double>(d, an, ROW_ANALYZE);
    cols_pass<double, COL_ANALYZE>(d, an, 0);

    if (precision == 32) return run<float>(d, nsv, T0, xi, steps, mode, tol, switch_tol, an.uh);
    return run<double>(d, nsv, T0, xi, steps, mode, tol, switch_tol, an.uh);
}
