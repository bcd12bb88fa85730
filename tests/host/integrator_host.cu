// Host build of the library's cell integrator (the same __host__ __device__
// code the CUDA kernels run), for CPU tests against the oracle.  Test
// infrastructure: compiled by tests/test_integrator_host.py, never linked into
// the library.
#include "../../paper_1201_5651_gb300/csrc/common.cuh"
#include "../../paper_1201_5651_gb300/csrc/integrator.cuh"
#include <cmath>

using namespace oots;

template <typename Real>
static void integrate_mono(double A, double b, double Nin, double c, double b0, double sigma0, double x0, double h,
                           double *out)
{
    SrcRate<Real> r;
    r.A = Real(A); r.b = Real(b); r.Nin = Real(Nin); r.p = Real(1); r.tab = -1;
    CellODE<Real> C;
    C.ns = 1; C.c = Real(c); C.b0 = Real(b0); C.r = &r; C.tabs = nullptr;
    const IntResult<Real> R = integrate_cell<Real, 1>(C, Real(x0), Real(h), Real(sigma0));
    out[0] = double(R.x);
    out[1] = double(R.IR);
    out[2] = double(R.lnfav);
}

// One monochromatic cell: F(x) = A (1 - exp(-b x)), dx/dt = -F + c (1 - x)^2,
// over h from x0; b0 > 0 also averages exp(-b0 x) (A1).  out: x(h), the
// recombinations per atom, ln <exp(-b0 x)>.  precision 0: double, 1: float.
extern "C" void oots_host_integrate_mono(int precision, double A, double b, double Nin, double c, double b0,
                                         double sigma0, double x0, double h, double *out)
{
    if (precision == 0) integrate_mono<double>(A, b, Nin, c, b0, sigma0, x0, h, out);
    else integrate_mono<float>(A, b, Nin, c, b0, sigma0, x0, h, out);
}

// A1 along one row lit by a plane-parallel monochromatic flux F, as the row
// kernel runs it: each cell integrates over dt with its entry column frozen and
// passes N_out = N_in - ln<f>/sigma0 on.  n, x (in/out) hold ncell values;
// returns the photons the row absorbed per unit area over nsteps steps.
extern "C" double oots_host_a1_row(int precision, int ncell, double F, double sigma0, double alpha, double dx,
                                   const double *n, double *x, double dt, int nsteps)
{
    double ions = 0.0;
    for (int s = 0; s < nsteps; s++) {
        double N = 0.0;
        for (int m = 0; m < ncell; m++) {
            const double A = F * std::exp(-sigma0 * N) / (n[m] * dx);
            double out[3];
            oots_host_integrate_mono(precision, A, sigma0 * n[m] * dx, N, alpha * n[m], sigma0 * n[m] * dx, sigma0,
                                     x[m], dt, out);
            double dtau = -out[2];
            if (!(dtau >= 0.0)) dtau = 0.0;
            ions += n[m] * dx * (x[m] - out[0]);
            x[m] = out[0];
            N += dtau / sigma0;
        }
    }
    return ions;
}

// ---- blackbody tables (tables.cpp builds them on the host, as the library does)
#include "../../paper_1201_5651_gb300/csrc/tables.h"
#include <vector>

template <typename Real> struct HostDevTable {
    std::vector<Real> coef, L, Nn;
    DevTable<Real> T;
    explicit HostDevTable(const HostTable &H)
        : coef(H.coef.begin(), H.coef.end()), L(H.L.begin(), H.L.end()), Nn(H.Nnode.begin(), H.Nnode.end())
    {
        T.coef = coef.data(); T.L = L.data(); T.Nnode = Nn.data();
        T.lnN_lo = Real(H.lnN_lo); T.dl = Real(H.dl); T.inv_dl = Real(1.0 / H.dl);
        T.N0 = Real(H.Nnode[0]); T.Nhi = Real(H.Nnode[H.K - 1]); T.a0 = Real(H.a0); T.K = H.K;
    }
};

// ln(P(N)/Q) of the blackbody table at T (precision 0: double, 1: float)
extern "C" void oots_host_table_lnp(int precision, double Tbb, double sigma0, const double *N, int m, double *out)
{
    const HostTable &H = host_table(1, Tbb, sigma0);
    if (precision == 0) {
        HostDevTable<double> D(H);
        for (int i = 0; i < m; i++) out[i] = tab_lnp(D.T, N[i]);
    } else {
        HostDevTable<float> D(H);
        for (int i = 0; i < m; i++) out[i] = double(tab_lnp(D.T, float(N[i])));
    }
}

template <typename Real>
static void integrate_bb(const HostTable &H, double A, double b, double Nin, double c, double sigma0, double x0,
                         double h, double *out)
{
    HostDevTable<Real> D(H);
    SrcRate<Real> r;
    r.A = Real(A); r.b = Real(b); r.Nin = Real(Nin); r.tab = 0;
    r.p = m_exp(tab_lnp(D.T, Real(Nin)));
    CellODE<Real> C;
    C.ns = 1; C.c = Real(c); C.b0 = Real(0); C.r = &r; C.tabs = &D.T;
    const IntResult<Real> R = integrate_cell<Real, 1>(C, Real(x0), Real(h), Real(sigma0));
    out[0] = double(R.x);
    out[1] = double(R.IR);
}

// One cell lit through the blackbody table: F(x) = A [P(Nin) - P(Nin + b x)]/Q
// with b = n ds (a column per unit x).  out: x(h), recombinations per atom.
extern "C" void oots_host_integrate_bb(int precision, double Tbb, double A, double b, double Nin, double c,
                                       double sigma0, double x0, double h, double *out)
{
    const HostTable &H = host_table(1, Tbb, sigma0);
    if (precision == 0) integrate_bb<double>(H, A, b, Nin, c, sigma0, x0, h, out);
    else integrate_bb<float>(H, A, b, Nin, c, sigma0, x0, h, out);
}

// ln P(Na + dN) - ln P(Na) of the blackbody table, by the library's stable
// difference (no cancellation for small dN)
extern "C" void oots_host_table_dlnp(int precision, double Tbb, double sigma0, const double *Na, const double *dN,
                                     int m, double *out)
{
    const HostTable &H = host_table(1, Tbb, sigma0);
    if (precision == 0) {
        HostDevTable<double> D(H);
        for (int i = 0; i < m; i++) out[i] = tab_dlnp(D.T, Na[i], dN[i]);
    } else {
        HostDevTable<float> D(H);
        for (int i = 0; i < m; i++) out[i] = double(tab_dlnp(D.T, float(Na[i]), float(dN[i])));
    }
}

// float-float running sum of m floats (the mixed path's column accumulation)
extern "C" double oots_host_ff_sum(const float *v, int m)
{
    ff s = ff_make(0.0f);
    for (int i = 0; i < m; i++) s = ff_add_f(s, v[i]);
    return double(s.hi) + double(s.lo);
}

// Monochromatic rate per H atom F(x) = A (1 - exp(-b x)) of one source for the
// cell (X, Y, Z) of an nx x ny x nz grid, from the library's src_rate: a point
// source at vertex v (Q photons/s) or, with plane = 1, a plane source (Q is
// then its flux).  N is the cell's entry column.
extern "C" double oots_host_rate_mono(int plane, const int *v, double Q, double sigma0, double dx, double n, int X,
                                      int Y, int Z, double N, double x)
{
    const int i = X >= v[0] ? X - v[0] : v[0] - 1 - X;
    const int j = Y >= v[1] ? Y - v[1] : v[1] - 1 - Y;
    const int k = Z >= v[2] ? Z - v[2] : v[2] - 1 - Z;
    const double qfac = plane ? Q / dx : Q / (4.0 * M_PI * dx * dx * dx);
    SrcRate<double> r;
    src_rate<double>(r, qfac, -1, sigma0, dx, n, plane != 0, i, j, k, N, nullptr);
    return -r.A * std::expm1(-r.b * x);
}
