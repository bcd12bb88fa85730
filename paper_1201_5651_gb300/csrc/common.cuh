// Device-side building blocks shared by the sweep and per-cell kernels:
// precision traits, float-float column arithmetic, rate tables and the
// per-cell rate parameters of the photon-conserving rate (Mackey 2012, Sect. 2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "oots_internal.h"

#define OOTS_HD __host__ __device__
// one out-of-line copy of a routine called from many sites (instruction-cache footprint)
#ifdef __CUDACC__
#define OOTS_NOINLINE __noinline__
#else
#define OOTS_NOINLINE __attribute__((noinline))
#endif

namespace oots {

// ---------------------------------------------------------------------------
// Float-float ("double-single") column accumulator for the mixed-precision
// path: an unevaluated sum hi + lo of two floats (about 48 significant bits),
// built from the error-free transformations of Knuth (two-sum) and Dekker
// (two-product via FMA).  Used only for the column density carried along rays.
// ---------------------------------------------------------------------------
struct ff { float hi, lo; };

OOTS_HD __forceinline__ ff ff_make(float a) { return ff{a, 0.0f}; }

OOTS_HD __forceinline__ ff ff_quick(float s, float e)
{
    float h = s + e;
    return ff{h, e - (h - s)};
}
OOTS_HD __forceinline__ ff ff_add(ff a, ff b)
{
    float s = a.hi + b.hi;
    float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    return ff_quick(s, e);
}
OOTS_HD __forceinline__ ff ff_add_f(ff a, float b)
{
    float s = a.hi + b;
    float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b - bb);
    e += a.lo;
    return ff_quick(s, e);
}
// a * f, exact product of the high part plus the low part's contribution
OOTS_HD __forceinline__ ff ff_mul_f(ff a, float f)
{
    float p = a.hi * f;
    float e = fmaf(a.hi, f, -p);
    e = fmaf(a.lo, f, e);
    return ff_quick(p, e);
}
// a / f with one correction step (remainder computed exactly)
OOTS_HD __forceinline__ ff ff_div_f(ff a, float f)
{
    float q1 = a.hi / f;
    float p = q1 * f;
    float pe = fmaf(q1, f, -p);
    // remainder r = a - q1 f computed as (a.hi - p) - pe + a.lo
    float r = ((a.hi - p) - pe) + a.lo;
    float q2 = r / f;
    return ff_quick(q1, q2);
}

// Column type per precision: FP64 path carries double, mixed path float-float.
template <typename Real> struct ColT;
template <> struct ColT<double> {
    typedef double type;
    static OOTS_HD __forceinline__ double zero() { return 0.0; }
    static OOTS_HD __forceinline__ double fma_w(double acc, double w, double N) { return fma(w, N, acc); }
    static OOTS_HD __forceinline__ double div(double a, double s) { return a / s; }
    static OOTS_HD __forceinline__ double add(double a, double d) { return a + d; }
    static OOTS_HD __forceinline__ double addc(double a, double b) { return a + b; }
    static OOTS_HD __forceinline__ double to_real(double a) { return a; }
    static OOTS_HD __forceinline__ double sub_r(double a, double b) { return a - b; }
    static OOTS_HD __forceinline__ double make(double hi, double) { return hi; }
    static OOTS_HD __forceinline__ double hi(double a) { return a; }
    static OOTS_HD __forceinline__ double lo(double) { return 0.0; }
};
template <> struct ColT<float> {
    typedef ff type;
    static OOTS_HD __forceinline__ ff zero() { return ff{0.0f, 0.0f}; }
    static OOTS_HD __forceinline__ ff fma_w(ff acc, float w, ff N) { return ff_add(acc, ff_mul_f(N, w)); }
    static OOTS_HD __forceinline__ ff div(ff a, float s) { return ff_div_f(a, s); }
    static OOTS_HD __forceinline__ ff add(ff a, float d) { return ff_add_f(a, d); }
    static OOTS_HD __forceinline__ ff addc(ff a, ff b) { return ff_add(a, b); }
    static OOTS_HD __forceinline__ float to_real(ff a) { return a.hi + a.lo; }
    // a - b rounded to one float (exact high-part difference for close columns)
    static OOTS_HD __forceinline__ float sub_r(ff a, ff b) { return (a.hi - b.hi) + (a.lo - b.lo); }
    static OOTS_HD __forceinline__ ff make(float hi, float lo) { return ff{hi, lo}; }
    static OOTS_HD __forceinline__ float hi(ff a) { return a.hi; }
    static OOTS_HD __forceinline__ float lo(ff a) { return a.lo; }
};

// ---------------------------------------------------------------------------
// Math wrappers: one spelling for both precisions.
// ---------------------------------------------------------------------------
OOTS_HD __forceinline__ double m_exp(double a) { return exp(a); }
OOTS_HD __forceinline__ float m_exp(float a) { return expf(a); }
OOTS_HD __forceinline__ double m_expm1(double a) { return expm1(a); }
OOTS_HD __forceinline__ float m_expm1(float a) { return expm1f(a); }
OOTS_HD __forceinline__ double m_log(double a) { return log(a); }
OOTS_HD __forceinline__ float m_log(float a) { return logf(a); }
OOTS_HD __forceinline__ double m_log1p(double a) { return log1p(a); }
OOTS_HD __forceinline__ float m_log1p(float a) { return log1pf(a); }
OOTS_HD __forceinline__ double m_sqrt(double a) { return sqrt(a); }
OOTS_HD __forceinline__ float m_sqrt(float a) { return sqrtf(a); }
OOTS_HD __forceinline__ double m_abs(double a) { return fabs(a); }
OOTS_HD __forceinline__ float m_abs(float a) { return fabsf(a); }
OOTS_HD __forceinline__ double m_min(double a, double b) { return fmin(a, b); }
OOTS_HD __forceinline__ float m_min(float a, float b) { return fminf(a, b); }
OOTS_HD __forceinline__ double m_max(double a, double b) { return fmax(a, b); }
OOTS_HD __forceinline__ float m_max(float a, float b) { return fmaxf(a, b); }

template <typename Real> struct RealLimits;
template <> struct RealLimits<double> {
    static OOTS_HD __forceinline__ double eps() { return 2.220446049250313e-16; }
    static OOTS_HD __forceinline__ double inf() { return HUGE_VAL; }
    static OOTS_HD __forceinline__ double tiny() { return 1e-300; }
};
template <> struct RealLimits<float> {
    static OOTS_HD __forceinline__ float eps() { return 1.1920929e-07f; }
    static OOTS_HD __forceinline__ float inf() { return HUGE_VALF; }
    static OOTS_HD __forceinline__ float tiny() { return 1e-37f; }
};

// ---------------------------------------------------------------------------
// Rate table of one source spectrum: ln(P/Q) at K log-spaced columns, as the
// monomial coefficients (in t = (ln N - ln N_k)/dl) of the quintic Hermite
// interpolant on every interval.  Below the first node P is linear in N; above
// the last node P = 0.
// ---------------------------------------------------------------------------
template <typename Real> struct DevTable {
    const Real *coef;   // (K-1) x 6
    const Real *L;      // K node values of ln(P/Q)
    const Real *Nnode;  // K node columns N_k
    Real lnN_lo, dl, inv_dl;
    Real N0, Nhi;       // first and last node column
    Real a0;            // 1 - P(N0)/Q
    int K;
};

template <typename Real>
OOTS_HD __forceinline__ int tab_interval(const DevTable<Real> &T, Real lnN)
{
    int k = (int)floor((lnN - T.lnN_lo) * T.inv_dl);
    return k < 0 ? 0 : (k > T.K - 2 ? T.K - 2 : k);
}

// ln(P(N)/Q); -inf above the table.
template <typename Real>
OOTS_HD OOTS_NOINLINE Real tab_lnp(const DevTable<Real> &T, Real N)
{
    if (N <= Real(0)) return Real(0);
    if (N < T.N0) return m_log1p(-T.a0 * (N / T.N0));
    if (N > T.Nhi) return -RealLimits<Real>::inf();
    Real lnN = m_log(N);
    int k = tab_interval(T, lnN);
    Real t = (lnN - (T.lnN_lo + Real(k) * T.dl)) * T.inv_dl;
    const Real *a = T.coef + 6 * k;
    return a[0] + t * (a[1] + t * (a[2] + t * (a[3] + t * (a[4] + t * a[5]))));
}

// Divided difference of the interval polynomial: (H(t2) - H(t1)) / (t2 - t1)
// as sum_m a_m (t2^m - t1^m)/(t2 - t1), evaluated without cancellation.
template <typename Real>
OOTS_HD __forceinline__ Real tab_dd(const Real *a, Real t1, Real t2)
{
    Real e = Real(1);        // (t2^1 - t1^1)/(t2 - t1)
    Real p1 = t1;            // t1^1
    Real s = a[1];
#pragma unroll
    for (int m = 2; m <= 5; m++) {
        e = t2 * e + p1;      // (t2^m - t1^m)/(t2 - t1)
        p1 *= t1;
        s += a[m] * e;
    }
    return s;
}

// d/dt of the interval polynomial at t
template <typename Real>
OOTS_HD __forceinline__ Real tab_dpoly(const Real *a, Real t)
{
    return a[1] + t * (Real(2) * a[2] + t * (Real(3) * a[3] + t * (Real(4) * a[4] + t * Real(5) * a[5])));
}

// ln P(Na + dN) - ln P(Na) (<= 0) from the exact increment dN, without
// cancellation: closed form on the linear piece below the table; inside the
// table the first and last partial intervals by divided differences and the
// whole intervals in between by node values.
template <typename Real>
OOTS_HD OOTS_NOINLINE Real tab_dlnp(const DevTable<Real> &T, Real Na, Real dN)
{
    if (!(dN > Real(0))) return Real(0);
    if (Na + dN > T.Nhi) return -RealLimits<Real>::inf();
    Real acc = Real(0);
    Real lo = Na, rem = dN;
    if (lo < T.N0) {
        Real piece = m_min(T.N0 - lo, rem);
        acc += m_log1p(-T.a0 * piece / (T.N0 - T.a0 * lo));
        if (piece >= rem) return acc;
        lo = T.N0;
        rem -= piece;
    }
    // first (possibly partial) interval
    Real lnlo = m_log(lo);
    int k = tab_interval(T, lnlo);
    Real Nk1 = T.Nnode[k + 1];
    if (Nk1 <= lo && k < T.K - 2) { k++; Nk1 = T.Nnode[k + 1]; }
    Real t1 = (lnlo - (T.lnN_lo + Real(k) * T.dl)) * T.inv_dl;
    if (lo == T.Nnode[k]) t1 = Real(0);
    Real piece = m_min(Nk1 - lo, rem);
    if (!(piece > Real(0))) piece = rem;
    Real dt = m_log1p(piece / lo) * T.inv_dl;
    acc += dt * tab_dd(T.coef + 6 * k, t1, t1 + dt);
    if (piece >= rem) return acc;
    rem -= piece;
    Real hi = Nk1 + rem;   // end column (the increment itself was used above)
    // whole intervals k+1 .. k2-1, then the partial interval k2
    Real lnhi = m_log(hi);
    int k2 = tab_interval(T, lnhi);
    if (k2 < k + 1) k2 = k + 1;
    if (T.Nnode[k2] > hi && k2 > k + 1) k2--;
    acc += T.L[k2] - T.L[k + 1];
    Real rem2 = (k2 == k + 1) ? rem : hi - T.Nnode[k2];
    if (rem2 > Real(0)) {
        Real dt2 = m_log1p(rem2 / T.Nnode[k2]) * T.inv_dl;
        acc += dt2 * tab_dd(T.coef + 6 * k2, Real(0), dt2);
    }
    return acc;
}

// d ln P / d N at N (for the slope of the rate at equilibrium)
template <typename Real>
OOTS_HD OOTS_NOINLINE Real tab_dlnp_dN(const DevTable<Real> &T, Real N)
{
    if (N < T.N0) return -T.a0 / (T.N0 - T.a0 * N);
    if (N > T.Nhi) return Real(0);
    Real lnN = m_log(N);
    int k = tab_interval(T, lnN);
    Real t = (lnN - (T.lnN_lo + Real(k) * T.dl)) * T.inv_dl;
    return tab_dpoly(T.coef + 6 * k, t) * T.inv_dl / N;
}

// ---------------------------------------------------------------------------
// Per-cell, per-source rate parameters (Sect. 2 rate; see the oracle header):
//   monochromatic: F(x) = A (1 - exp(-b x)),   A = R_in/(n V_sh), b = sigma0 n ds
//   tabulated:     F(x) = A p [1 - P(Nin + b x)/P(Nin)], A = Q/(n V_sh), b = n ds,
//                  p = P(Nin)/Q
// ---------------------------------------------------------------------------
template <typename Real> struct SrcRate {
    Real A, b, Nin, p;
    int tab;              // -1: monochromatic; otherwise index of the table
};

// Rate parameters of one source for the cell (i,j,k) of its octant (vertex
// at the origin) with entry column N: qfac = Q / (4 pi dx^3); the shell is
// 4 pi r^2 ds with r^2 ds in units of dx^3.  A plane source (plane = true;
// i, j, k unused) has ds = dx and shares the photons it loses over the cell's
// volume per unit face area, dx: qfac = F / dx.  with_p = false leaves p of a
// tabulated source to the caller.
template <typename Real>
OOTS_HD __forceinline__ void src_rate(SrcRate<Real> &r, Real qfac, int tab, Real sigma0, Real dx, Real n, bool plane,
                                      int i, int j, int k, Real N, const DevTable<Real> *tabs, bool with_p = true)
{
    Real sf = Real(1), den = n;   // den = n V_sh in units of 4 pi dx^3 (point) or dx (plane)
    if (!plane) {
        const Real c0 = Real(i) + Real(0.5), c1 = Real(j) + Real(0.5), c2 = Real(k) + Real(0.5);
        const Real r2 = c0 * c0 + c1 * c1 + c2 * c2;
        sf = m_sqrt(r2) / m_max(c0, m_max(c1, c2));
        den = n * r2 * sf;
    }
    r.Nin = N;
    r.tab = tab;
    if (tab < 0) {
        // Q e^{-sigma0 N} / (n V_sh)
        r.A = qfac * m_exp(-sigma0 * N) / den;
        r.b = sigma0 * n * dx * sf;
        r.p = Real(1);
    } else {
        r.A = qfac / den;
        r.b = n * dx * sf;
        if (with_p) r.p = m_exp(tab_lnp(tabs[tab], N));
    }
}

} // namespace oots
