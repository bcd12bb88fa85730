// Per-cell integrator of the neutral-fraction ODE (Mackey 2012, Eq. 2 with the
// temperature fixed and collisional ionisation off):
//
//     dx/dt = f(x) = -F(x) + c (1 - x)^2,   c = alpha_B n,
//
// where F(x) = sum_s F_s(x) is the photon-conserving photoionisation rate per
// H atom with the entry columns frozen and the cell's own optical depth
// evolving with x.  f is convex and strictly decreasing on [0,1], so x moves
// monotonically to the unique root x_eq.
//
// Method (time-to-state inversion): with u = ln((x - x_eq)/(x0 - x_eq)),
// du/dt = -D(u) where D = -(f(x_eq + d) - f(x_eq))/d > 0 (d = x - x_eq) is the
// secant slope, evaluated from difference forms without cancellation.  The
// elapsed time T(u) = int_u^0 du'/D(u') is accumulated over Gauss-Legendre
// panels in u; the panel in which T reaches h is inverted through the
// Legendre interpolant of 1/D on its nodes (no further evaluations).  Close
// to equilibrium (|d| small against the scales on which F and the
// recombination term bend) T(u) = T_t + (u_t - u)/D_inf + R(e^u) with R smooth
// in w = e^u, integrated by one more Gauss rule in w.  The time integrals of
// the recombination term (for the photon budget) and of exp(-b0 x) (for the
// time-averaged attenuation of A1, Eq. 3) are accumulated on the same nodes.
#pragma once
#include "common.cuh"

namespace oots {

// Gauss-Legendre rules on [-1, 1] (nodes and weights in the working precision).
template <int G> struct GL;
template <> struct GL<4> {
    template <typename Real> static OOTS_HD __forceinline__ Real x(int i) {
        return i == 0 ? Real(-0.8611363115940526) : i == 1 ? Real(-0.3399810435848563) : i == 2 ? Real(0.3399810435848563) : Real(0.8611363115940526);
    }
    template <typename Real> static OOTS_HD __forceinline__ Real w(int i) {
        return (i == 0 || i == 3) ? Real(0.3478548451374538) : Real(0.6521451548625461);
    }
};
template <> struct GL<8> {
    template <typename Real> static OOTS_HD __forceinline__ Real x(int i) {
        return i == 0 ? Real(-0.9602898564975363) : i == 1 ? Real(-0.7966664774136267) : i == 2 ? Real(-0.5255324099163290)
             : i == 3 ? Real(-0.1834346424956498) : i == 4 ? Real(0.1834346424956498) : i == 5 ? Real(0.5255324099163290)
             : i == 6 ? Real(0.7966664774136267) : Real(0.9602898564975363);
    }
    template <typename Real> static OOTS_HD __forceinline__ Real w(int i) {
        return (i == 0 || i == 7) ? Real(0.1012285362903763) : (i == 1 || i == 6) ? Real(0.2223810344533745)
             : (i == 2 || i == 5) ? Real(0.3137066458778873) : Real(0.3626837833783620);
    }
};

// Legendre polynomials P_0..P_{n-1} at s by the three-term recurrence.
template <typename Real, int N>
OOTS_HD __forceinline__ void legendre(Real s, Real *P)
{
    P[0] = Real(1);
    if (N > 1) P[1] = s;
#pragma unroll
    for (int n = 1; n + 1 < N; n++) P[n + 1] = (Real(2 * n + 1) * s * P[n] - Real(n) * P[n - 1]) / Real(n + 1);
}

// Legendre coefficients of the degree G-1 interpolant through G Gauss nodal values.
template <typename Real, int G>
OOTS_HD __forceinline__ void leg_coeffs(const Real *v, Real *c)
{
#pragma unroll
    for (int n = 0; n < G; n++) c[n] = Real(0);
#pragma unroll
    for (int g = 0; g < G; g++) {
        Real P[G];
        legendre<Real, G>(GL<G>::template x<Real>(g), P);
        Real wv = GL<G>::template w<Real>(g) * v[g];
#pragma unroll
        for (int n = 0; n < G; n++) c[n] += wv * P[n];
    }
#pragma unroll
    for (int n = 0; n < G; n++) c[n] *= Real(2 * n + 1) * Real(0.5);
}

// int_s^1 of the interpolant (Legendre coefficients c) and its value at s.
// The interpolant has degree G-1, so the G-point Gauss rule on [s, 1] gives its
// integral exactly, with no cancellation as s -> 1.
template <typename Real, int G>
OOTS_HD __forceinline__ Real leg_eval(const Real *c, Real t)
{
    Real P[G];
    legendre<Real, G>(t, P);
    Real v = Real(0);
#pragma unroll
    for (int n = 0; n < G; n++) v += c[n] * P[n];
    return v;
}

template <typename Real, int G>
OOTS_HD __forceinline__ void leg_tail(const Real *c, Real s, Real *integral, Real *value)
{
    const Real hw = Real(0.5) * (Real(1) - s), mid = Real(0.5) * (Real(1) + s);
    Real I = Real(0);
#pragma unroll
    for (int g = 0; g < G; g++) I += GL<G>::template w<Real>(g) * leg_eval<Real, G>(c, mid + hw * GL<G>::template x<Real>(g));
    *integral = hw * I;
    *value = leg_eval<Real, G>(c, s);
}

// Everything the integrator needs about one cell.
template <typename Real> struct CellODE {
    int ns;
    Real c;                      // alpha n
    Real b0;                     // sigma0 n ds of the source traced by A1 (0: not needed)
    SrcRate<Real> *r;            // ns entries
    const DevTable<Real> *tabs;  // table of every tabulated source
};

template <typename Real> struct IntResult {
    Real x;      // x(h)
    Real IR;     // int_0^h c (1-x)^2 dt: recombinations per H atom
    Real lnfav;  // ln <exp(-b0 x)> over the step
};

// One source's term of F(x) and F'(x), added to s and d
template <typename Real>
OOTS_HD __forceinline__ void src_F_term(const SrcRate<Real> &r, const DevTable<Real> *tabs, Real x, Real &s, Real &d)
{
    if (!(r.A > Real(0))) return;
    if (r.tab < 0) {
        Real e = m_expm1(-r.b * x);          // e^{-bx} - 1
        s += -r.A * e;
        d += r.A * r.b * (Real(1) + e);
    } else {
        const DevTable<Real> &T = tabs[r.tab];
        Real dl = tab_dlnp(T, r.Nin, r.b * x);
        s += -r.A * r.p * m_expm1(dl);
        Real px = r.p * m_exp(dl);            // P(Nin + b x)/Q
        if (px > Real(0)) d += -r.A * px * r.b * tab_dlnp_dN(T, r.Nin + r.b * x);
    }
}

// F(x) and F'(x)
template <typename Real, int NSMAX = MAX_SRC>
OOTS_HD OOTS_NOINLINE void ode_F(const CellODE<Real> &C, Real x, Real *F, Real *dF)
{
    Real s = Real(0), d = Real(0);
    for (int i = 0; i < NSMAX && i < C.ns; i++) src_F_term(C.r[i], C.tabs, x, s, d);
    *F = s;
    *dF = d;
}

// Per-source values at the root, used by the secant slope:
//   lne = ln of the transmitted fraction at the root (monochromatic: -b xe;
//   tabulated: ln(P(Ne)/Q)), Ne = entry column + b xe (tabulated only).
template <typename Real> struct SrcEq { Real lne; Real Ne; };

// D = (F(xe + d) - F(xe))/d + c (2 (1 - xe) - d), d != 0, from difference
// forms that keep full relative precision for small |d| and cannot overflow
// for large |d| (every product below is a transmitted fraction <= 1).
template <typename Real, int NSMAX = MAX_SRC>
OOTS_HD OOTS_NOINLINE Real ode_D(const CellODE<Real> &C, const SrcEq<Real> *Q, Real xe, Real d)
{
    Real s = Real(0);
    const bool tiny = m_abs(d) < RealLimits<Real>::tiny() * Real(1e10);
    for (int i = 0; i < NSMAX && i < C.ns; i++) {
        const SrcRate<Real> &r = C.r[i];
        if (!(r.A > Real(0))) continue;
        if (r.tab < 0) {
            // A b e^{-b xe} (1 - e^{-z})/z, z = b d, the ratio formed first (no underflow)
            const Real z = r.b * d;
            if (z > Real(-20)) {
                const Real q = (z != Real(0) && !tiny) ? -m_expm1(-z) / z : Real(1);
                s += r.A * r.b * m_exp(Q[i].lne) * q;
            } else {
                s += r.A * (m_exp(Q[i].lne) - m_exp(Q[i].lne - z)) / d;
            }
        } else {
            const DevTable<Real> &T = C.tabs[r.tab];
            Real dl = Real(0);
            if (!tiny) dl = d > Real(0) ? tab_dlnp(T, Q[i].Ne, r.b * d)              // ln P(Ne + b d) - ln P(Ne)
                                        : tab_dlnp(T, Q[i].Ne + r.b * d, -r.b * d);  // ln P(Ne) - ln P(Ne + b d)
            if (dl == Real(0)) {
                // limit d -> 0: -A b P(Ne)/Q d ln P/dN
                const Real pe = m_exp(Q[i].lne);
                if (pe > Real(0)) s += -r.A * pe * r.b * tab_dlnp_dN(T, Q[i].Ne);
            } else if (d > Real(0)) {
                s += r.A * m_exp(Q[i].lne) * (-m_expm1(dl)) / d;
            } else {
                s += -r.A * m_exp(Q[i].lne - dl) * (-m_expm1(dl)) / d;   // -(P(Ne+bd) - P(Ne))/(Q d)
            }
        }
    }
    return s + C.c * (Real(2) * (Real(1) - xe) - d);
}

template <typename Real> struct IntCfg;
template <> struct IntCfg<double> {
    enum { G = 8 };
    static OOTS_HD double umax() { return 40.0; }
    static OOTS_HD double tolq() { return 1e-14; }
    static OOTS_HD double zlin() { return 1e-6; }    // linearised step allowed below this h|f'|
};
template <> struct IntCfg<float> {
    enum { G = 4 };
    static OOTS_HD float umax() { return 20.0f; }
    static OOTS_HD float tolq() { return 1e-6f; }
    static OOTS_HD float zlin() { return 3e-3f; }
};

template <typename Real, int NSMAX>
OOTS_HD Real attenuation_average(const CellODE<Real> &C, const SrcEq<Real> *Q, Real xe, Real d0, Real Dinf,
                                 Real h, Real ustar, Real ut, bool in_panels, Real wt);

// Root of the convex, decreasing right-hand side by Newton inside the
// bracket [lo, hi], from xk (with f, F and f' there): from the right of the
// root the first step lands left of it, and from the left Newton increases
// monotonically to it.  f is a difference of two terms, so it is known only to
// about eps times their size: Newton also stops once |f| is inside that
// rounding band (the iterate would otherwise jitter inside it without meeting
// the step test).
template <typename Real, int NSMAX>
OOTS_HD Real newton_root(const CellODE<Real> &C, Real lo, Real hi, Real xk, Real fk, Real Fk, Real dfk)
{
    Real xe = xk;
    for (int it = 0; it < 60; it++) {
        if (m_abs(fk) <= Real(32) * RealLimits<Real>::eps() * (m_abs(Fk) + C.c * (Real(1) - xk) * (Real(1) - xk))) break;
        if (fk > Real(0)) lo = m_max(lo, xk); else hi = m_min(hi, xk);
        Real xn = (dfk < Real(0)) ? xk - fk / dfk : Real(0.5) * (lo + hi);
        if (!(xn >= lo && xn <= hi)) xn = Real(0.5) * (lo + hi);
        const bool done = m_abs(xn - xk) <= Real(4) * RealLimits<Real>::eps() * m_max(xn, RealLimits<Real>::tiny())
                       || (hi - lo) <= Real(4) * RealLimits<Real>::eps() * m_max(hi, RealLimits<Real>::tiny());
        xk = xn;
        Real dFk;
        ode_F<Real, NSMAX>(C, xk, &Fk, &dFk);
        fk = -Fk + C.c * (Real(1) - xk) * (Real(1) - xk);
        dfk = -dFk - Real(2) * C.c * (Real(1) - xk);
        xe = xk;
        if (done) break;
    }
    return xe;
}

// Evaluators of the general path.
//  - root(C, x0, f0, F0, dF0): the root x_eq of f.
//  - eval<N>(node, invD, dv): fills invD[l] = 1/D and dv[l] = d at the N
//    quadrature nodes l = 0..N-1, where node(l, d) returns 1/D at node l and
//    sets its deviation d.
// The sequential form runs Newton from x0 and loops over the nodes.  The group
// form (a half or whole warp per cell) brackets the root with one sample per
// lane at once and gives node l to lane l, broadcasting the values: a panel
// costs one evaluation of latency and the root search a scan plus a short
// polish.
struct SeqEval {
    static constexpr bool attenuation = true;    // A1's time-averaged attenuation when b0 > 0
    template <typename Real, int NSMAX>
    OOTS_HD Real root(const CellODE<Real> &C, Real x0, Real f0, Real F0, Real dF0) const
    {
        const Real lo = f0 > Real(0) ? x0 : Real(0), hi = f0 > Real(0) ? Real(1) : x0;
        return newton_root<Real, NSMAX>(C, lo, hi, x0, f0, F0, -dF0 - Real(2) * C.c * (Real(1) - x0));
    }
    template <int N, typename Real, typename Node>
    OOTS_HD __forceinline__ void eval(const Node &node, Real *invD, Real *dv) const
    {
#pragma unroll
        for (int l = 0; l < N; l++) invD[l] = node(l, dv[l]);
    }
};
#ifdef __CUDACC__
template <int W> struct GroupEval {
    static_assert(W == 16 || W == 32, "half warp or whole warp");
    static constexpr bool attenuation = false;   // integration passes only (b0 = 0)
    int lane;          // lane within the group, 0..W-1
    int base;          // first lane of the group within its warp
    unsigned mask;     // the group's lanes
    template <typename Real> __device__ __forceinline__ Real bcast(Real v, int l) const
    {
        return __shfl_sync(mask, v, base + l);
    }
    // Lane l samples f at a point of the bracket, ascending in x with l and
    // geometric towards the end the root lies away from (x for a root below
    // x0, 1 - x for a root above it) over nine decades; f > 0 exactly left
    // of the root, so the ballot of f > 0 marks the lanes below it.  Newton
    // polishes from the left end of the sign change.
    template <typename Real, int NSMAX>
    __device__ Real root(const CellODE<Real> &C, Real x0, Real f0, Real F0, Real dF0) const
    {
        const bool above = f0 > Real(0);                     // root in (x0, 1]
        const Real span = above ? Real(1) - x0 : x0;
        const Real step = Real(-20.7233) / Real(W);          // ln(1e-9) over the group's samples
        const Real p = above ? Real(1) - span * m_exp(step * Real(lane + 1)) : span * m_exp(step * Real(W - lane));
        Real Fp, dFp;
        ode_F<Real, NSMAX>(C, p, &Fp, &dFp);
        const Real fp = -Fp + C.c * (Real(1) - p) * (Real(1) - p);
        const Real dfp = -dFp - Real(2) * C.c * (Real(1) - p);
        const unsigned all = W == 32 ? 0xffffffffu : 0xffffu;
        const unsigned pos = (__ballot_sync(mask, fp > Real(0)) >> base) & all;
        const int j = (pos == all) ? W : __ffs(~pos) - 1;     // first sample right of the root
        // bracket [lo, hi] and the starting end
        const int lj = j & (W - 1), ljm = (j + W - 1) & (W - 1);
        const Real pj = bcast(p, lj), pjm = bcast(p, ljm);
        const Real fjm = bcast(fp, ljm), Fjm = bcast(Fp, ljm), dfjm = bcast(dfp, ljm);
        const Real fj = bcast(fp, lj), Fj = bcast(Fp, lj), dfj = bcast(dfp, lj);
        const Real lo = j > 0 ? pjm : (above ? x0 : Real(0));
        const Real hi = j < W ? pj : (above ? Real(1) : x0);
        if (j > 0) return newton_root<Real, NSMAX>(C, lo, hi, pjm, fjm, Fjm, dfjm);
        if (above) return newton_root<Real, NSMAX>(C, lo, hi, x0, f0, F0, -dF0 - Real(2) * C.c * (Real(1) - x0));
        return newton_root<Real, NSMAX>(C, lo, hi, pj, fj, Fj, dfj);
    }
    template <int N, typename Real, typename Node>
    __device__ __forceinline__ void eval(const Node &node, Real *invD, Real *dv) const
    {
        static_assert(N <= W, "one node per lane");
        Real mi = Real(0), md = Real(0);
        if (lane < N) mi = node(lane, md);
#pragma unroll
        for (int l = 0; l < N; l++) {
            invD[l] = bcast(mi, l);
            dv[l] = bcast(md, l);
        }
    }
};
// lanes per cell of the general pass: the FP32 panel's 3G = 12 nodes fit a
// half warp (two cells per warp); FP64's 24 take a whole warp
template <typename Real> struct GroupWidth { enum { value = 3 * IntCfg<Real>::G <= 16 ? 16 : 32 }; };
#endif

// Per-source values at the root x_eq and the slope there: Dinf = -f'(x_eq),
// and bmax, the largest optical depth scale per unit x (the rate bends on
// |d| ~ 1/bmax).
template <typename Real, int NSMAX>
OOTS_HD void root_slope(const CellODE<Real> &C, Real xe, Real sigma0, SrcEq<Real> *Q, Real &Dinf, Real &bmax)
{
    bmax = Real(0);
    Dinf = Real(2) * C.c * (Real(1) - xe);
    for (int i = 0; i < NSMAX && i < C.ns; i++) {
        const SrcRate<Real> &r = C.r[i];
        Q[i].lne = -RealLimits<Real>::inf();
        Q[i].Ne = Real(0);
        if (!(r.A > Real(0))) continue;
        if (r.tab < 0) {
            Q[i].lne = -r.b * xe;
            Dinf += r.A * r.b * m_exp(Q[i].lne);
            bmax = m_max(bmax, r.b);
        } else {
            const DevTable<Real> &T = C.tabs[r.tab];
            Q[i].Ne = r.Nin + r.b * xe;
            Q[i].lne = m_log(r.p) + tab_dlnp(T, r.Nin, r.b * xe);
            Real pe = m_exp(Q[i].lne);
            if (pe > Real(0)) Dinf += -r.A * pe * r.b * tab_dlnp_dN(T, Q[i].Ne);
            bmax = m_max(bmax, sigma0 * r.b);
        }
    }
}

// Already next to the root (|d0| = |x0 - x_eq| far below both bending scales):
// the linearised solution about x_eq, d(t) = d0 e^{-Dinf t}.  Returns false
// when the state is not that close.
template <typename Real>
OOTS_HD bool near_root_solution(const CellODE<Real> &C, Real xe, Real d0, Real Dinf, Real bmax, Real h,
                                IntResult<Real> &R)
{
    const Real ad0 = m_abs(d0);
    if (!(bmax * ad0 <= IntCfg<Real>::zlin() && ad0 <= IntCfg<Real>::zlin() * (Real(1) - xe) && C.b0 == Real(0)))
        return false;
    const Real e = m_exp(-Dinf * h);
    R.x = xe + d0 * e;
    const Real one = Real(1) - xe;
    // int c (1 - xe - d)^2 dt = c one^2 h - 2 c one d0 (1 - e)/Dinf + c d0^2 (1 - e^2)/(2 Dinf)
    const Real g1 = (Dinf * h > Real(1e-6)) ? -m_expm1(-Dinf * h) / Dinf : h;
    const Real g2 = (Dinf * h > Real(1e-6)) ? -m_expm1(Real(-2) * Dinf * h) / (Real(2) * Dinf) : h;
    R.IR = C.c * (one * one * h - Real(2) * one * d0 * g1 + d0 * d0 * g2);
    return true;
}

// First part of the integration: the closed forms.  Returns true when the
// cell is done (photon-free, at its root, or slow enough for the linearised
// step); otherwise F(x0), F'(x0) and f(x0) are left for the general part.
// have_F: F0 and dF0 already hold F(x0) and F'(x0).
template <typename Real, int NSMAX = MAX_SRC>
OOTS_HD bool integrate_prelude(const CellODE<Real> &C, Real x0, Real h, Real sigma0, IntResult<Real> &R,
                               Real &F0, Real &dF0, Real &f0, bool have_F = false)
{
    constexpr int G = IntCfg<Real>::G;
    R.x = x0;
    R.IR = Real(0);
    R.lnfav = -C.b0 * x0;
    if (!have_F) F0 = dF0 = Real(0);
    f0 = Real(0);
    if (!(h > Real(0))) return true;

    // photon-free cell: du/dt = -c u^2, u = 1 - x (closed form).  A source
    // counts only if it can move x by more than a thousandth of the rounding
    // over h: its rate is at most A b x (monochromatic) or A p sigma0 b x
    // (tabulated: no cross-section exceeds sigma0), so below that bound its
    // effect is dropped.  This also keeps subnormal rates (a cell hundreds of
    // optical depths down a row, with no recombinations to hold it) out of the
    // quadrature, whose 1/D they would overflow.  The exception is A1 with
    // recombinations (b0 > 0, c > 0): the attenuation average below is a fixed
    // Gauss rule on the recombination trajectory, exact only when x stays put,
    // so any nonzero rate keeps the full integration and its exact average.
    bool lit = false;
    const bool keep_any = C.b0 > Real(0) && C.c > Real(0);
    for (int i = 0; i < NSMAX && i < C.ns; i++) {
        const SrcRate<Real> &r = C.r[i];
        const Real amp = r.tab < 0 ? r.A * r.b : r.A * r.p * sigma0 * r.b;
        lit |= (amp * h > Real(1e-3) * RealLimits<Real>::eps()) || (keep_any && r.A > Real(0));
    }
    if (!lit) {
        Real u0 = Real(1) - x0;
        Real u = u0 / (Real(1) + C.c * u0 * h);
        R.x = Real(1) - u;
        R.IR = u0 - u;
        if (C.b0 > Real(0)) {
            // x rises monotonically from x0: average exp(-b0 (x(t) - x0)) by
            // Gauss-Legendre in t on the closed-form trajectory
            Real acc = Real(0);
#pragma unroll
            for (int g = 0; g < G; g++) {
                Real t = Real(0.5) * h * (Real(1) + GL<G>::template x<Real>(g));
                Real ut = u0 / (Real(1) + C.c * u0 * t);
                acc += GL<G>::template w<Real>(g) * Real(0.5) * m_exp(-C.b0 * (u0 - ut));
            }
            R.lnfav = -C.b0 * x0 + m_log(acc);
        }
        return true;
    }

    if (!have_F) ode_F<Real, NSMAX>(C, x0, &F0, &dF0);
    f0 = -F0 + C.c * (Real(1) - x0) * (Real(1) - x0);
    // at the root to within the rounding of f: x stays
    if (m_abs(f0) <= Real(32) * RealLimits<Real>::eps() * (m_abs(F0) + C.c * (Real(1) - x0) * (Real(1) - x0))) {
        R.IR = h * C.c * (Real(1) - x0) * (Real(1) - x0);
        return true;
    }
    // slow cells: when h |f'| is small and the step moves x by much less than
    // the scales on which f bends (1/b of every source, and 1 - x for the
    // recombination term), the linearised solution x0 + f0 (e^{h f'} - 1)/f'
    // is exact to the working tolerance; IR by the midpoint rule
    if (C.b0 == Real(0)) {
        const Real df0 = -dF0 - Real(2) * C.c * (Real(1) - x0);
        const Real z = h * df0;
        if (m_abs(z) <= IntCfg<Real>::zlin()) {
            const Real phi = (m_abs(z) > Real(1e-8)) ? m_expm1(z) / z : Real(1) + Real(0.5) * z;
            const Real dx = h * f0 * phi;
            Real bm = Real(0);
            for (int i = 0; i < NSMAX && i < C.ns; i++)
                if (C.r[i].A > Real(0)) bm = m_max(bm, C.r[i].tab < 0 ? C.r[i].b : sigma0 * C.r[i].b);
            const Real adx = m_abs(dx);
            // photoionisation bends on 1/b; the recombination term's curvature 2c
            // changes the increment by ~ c h dx relative
            if (bm * adx <= IntCfg<Real>::zlin() && C.c * h * adx <= IntCfg<Real>::zlin() * IntCfg<Real>::zlin() &&
                x0 + dx >= Real(0) && x0 + dx <= Real(1)) {
                R.x = x0 + dx;
                const Real xm = x0 + Real(0.5) * dx;
                R.IR = h * C.c * (Real(1) - xm) * (Real(1) - xm);
                return true;
            }
        }
        // near the root: when one Newton step puts x_eq within both bending
        // scales of x0, up to three Newton steps find it (f is smooth there)
        // and the linearised solution about it finishes the cell
        Real bm = Real(0);
        for (int i = 0; i < NSMAX && i < C.ns; i++)
            if (C.r[i].A > Real(0)) bm = m_max(bm, C.r[i].tab < 0 ? C.r[i].b : sigma0 * C.r[i].b);
        const Real est = df0 < Real(0) ? m_abs(f0 / df0) : RealLimits<Real>::inf();
        if (bm * est <= IntCfg<Real>::zlin() && est <= IntCfg<Real>::zlin() * (Real(1) - x0 + est)) {
            Real xk = x0, fk = f0, Fk = F0, dfk = df0;
            bool conv = false;
            for (int it = 0; it < 3 && dfk < Real(0); it++) {
                xk = m_min(m_max(xk - fk / dfk, Real(0)), Real(1));
                Real dFk;
                ode_F<Real, NSMAX>(C, xk, &Fk, &dFk);
                fk = -Fk + C.c * (Real(1) - xk) * (Real(1) - xk);
                dfk = -dFk - Real(2) * C.c * (Real(1) - xk);
                if (m_abs(fk) <= Real(32) * RealLimits<Real>::eps() * (m_abs(Fk) + C.c * (Real(1) - xk) * (Real(1) - xk))) {
                    conv = true;
                    break;
                }
            }
            if (conv) {
                SrcEq<Real> Q[NSMAX];
                Real Dinf, bmax;
                root_slope<Real, NSMAX>(C, xk, sigma0, Q, Dinf, bmax);
                if (near_root_solution<Real>(C, xk, x0 - xk, Dinf, bmax, h, R)) return true;
                R.x = x0;          // not close enough: leave it to the general part
                R.IR = Real(0);
            }
        }
    }
    return false;
}

// Second part: the root, then the time-to-state quadrature (see the header).
// R carries the prelude's defaults; ev evaluates the quadrature nodes.
#pragma nv_exec_check_disable
template <typename Real, int NSMAX, typename Eval>
OOTS_HD IntResult<Real> integrate_general(const CellODE<Real> &C, Real x0, Real h, Real sigma0, IntResult<Real> R,
                                          Real F0, Real dF0, Real f0, const Eval &ev)
{
    constexpr int G = IntCfg<Real>::G;
    const Real xe = ev.template root<Real, NSMAX>(C, x0, f0, F0, dF0);
    Real d0 = x0 - xe;
    if (d0 == Real(0)) {
        R.IR = h * C.c * (Real(1) - x0) * (Real(1) - x0);
        return R;
    }

    // per-source values at the root and the slope at the root
    SrcEq<Real> Q[NSMAX];
    Real Dinf, bmax;
    root_slope<Real, NSMAX>(C, xe, sigma0, Q, Dinf, bmax);
    const Real ad0 = m_abs(d0);
    if (near_root_solution<Real>(C, xe, d0, Dinf, bmax, h, R)) return R;
    // start of the near-equilibrium tail in w = e^u: the secant slope bends on
    // |d| ~ 1/bmax (photoionisation) and |d| ~ 1 - xe (recombination)
    Real wt = Real(1);
    if (bmax * ad0 > Real(0.5)) wt = Real(0.5) / (bmax * ad0);
    if (Real(0.5) * (Real(1) - xe) < wt * ad0) wt = Real(0.5) * (Real(1) - xe) / ad0;
    Real ut = m_log(wt);
    // when the tail would start deeper than umax, |d| is already below the
    // working precision there: start it at -umax and drop its smooth remainder
    const bool clamped = ut < -IntCfg<Real>::umax();
    if (clamped) ut = -IntCfg<Real>::umax();

    Real T = Real(0), IR = Real(0);
    Real uk = Real(0);
    bool found = false;
    Real ustar = Real(0);
    // adaptive panels in u: a panel is accepted when its Gauss sum agrees with
    // the sum over its two halves to tolq * h; the halves are then used
    // near u = 0 the rate bends on du ~ 1/(b |d0|) whenever the starting state
    // lies in a source's thin-to-saturated transition (b x0 < 40): start the
    // panels at that scale (they double after each accepted panel)
    Real du = Real(1);
    for (int i = 0; i < NSMAX && i < C.ns; i++) {
        if (!(C.r[i].A > Real(0))) continue;
        const Real bi = C.r[i].tab < 0 ? C.r[i].b : sigma0 * C.r[i].b;
        if (bi * x0 < Real(40) && bi * ad0 > Real(0.25)) du = m_min(du, Real(0.25) / (bi * ad0));
    }
    const Real tolq = IntCfg<Real>::tolq() * h;
    int npan = 0;
    while (uk > ut && npan < 400) {
        Real ua = uk - du;
        if (ua < ut) ua = ut;
        Real um = Real(0.5) * (uk + ua);
        // nodal values of 1/D on both halves (nodes 0..G-1: upper half [um, uk];
        // G..2G-1: lower half [ua, um]) and on the whole panel (2G..3G-1)
        Real iv[3 * G], dvv[3 * G];
        {
            const Real ukc = uk, uac = ua, umc = um;
            auto node = [&](int l, Real &d) {
                const int part = l / G, g = l - part * G;
                const Real lo = part == 0 ? umc : uac, hi = part == 1 ? umc : ukc;
                const Real u = Real(0.5) * (hi + lo) + Real(0.5) * (hi - lo) * GL<G>::template x<Real>(g);
                d = d0 * m_exp(u);
                return Real(1) / ode_D<Real, NSMAX>(C, Q, xe, d);
            };
            ev.template eval<3 * G>(node, iv, dvv);
        }
        Real vD[2][G], vR[2][G], Ih[2];
        for (int hh = 0; hh < 2; hh++) {
            const Real lo = hh ? ua : um, hi = hh ? um : uk;     // hh = 0: upper half [um, uk]
            const Real hw = Real(0.5) * (hi - lo);
            Ih[hh] = Real(0);
#pragma unroll
            for (int g = 0; g < G; g++) {
                const Real invD = iv[hh * G + g];
                const Real xi = xe + dvv[hh * G + g];
                vD[hh][g] = invD;
                vR[hh][g] = C.c * (Real(1) - xi) * (Real(1) - xi) * invD;
                Ih[hh] += GL<G>::template w<Real>(g) * hw * invD;
            }
        }
        // the whole panel by one Gauss sum, to estimate the error of the halves
        Real Ifull = Real(0);
        {
            const Real hw = Real(0.5) * (uk - ua);
#pragma unroll
            for (int g = 0; g < G; g++) Ifull += GL<G>::template w<Real>(g) * hw * iv[2 * G + g];
        }
        npan++;
        const Real err = m_abs(Ifull - (Ih[0] + Ih[1]));
        if (err > tolq && (uk - ua) > Real(1e-9)) {
            du = Real(0.5) * (uk - ua);
            continue;
        }
        // accepted: walk the upper half, then the lower half
        for (int hh = 0; hh < 2 && !found; hh++) {
            const Real lo = hh ? ua : um, hi = hh ? um : uk;
            const Real hw = Real(0.5) * (hi - lo), mid = Real(0.5) * (hi + lo);
            if (T + Ih[hh] >= h) {
                // invert within the half: s in [-1, 1] maps to u = mid + hw s;
                // T(s) = T + hw * int_s^1 (1/D); solve T(s) = h
                Real cD[G], cR[G];
                leg_coeffs<Real, G>(vD[hh], cD);
                leg_coeffs<Real, G>(vR[hh], cR);
                Real s = Real(1) - Real(2) * (h - T) / Ih[hh];
                if (s < Real(-1)) s = Real(-1);
                Real slo = Real(-1), shi = Real(1);
                for (int it = 0; it < 60; it++) {
                    Real I, v;
                    leg_tail<Real, G>(cD, s, &I, &v);
                    Real g = T + hw * I - h;            // decreasing in s, g(-1) >= 0 > g(1)
                    if (g == Real(0)) break;
                    if (g > Real(0)) slo = s; else shi = s;
                    Real sn = s + g / (hw * v);
                    if (!(sn > slo && sn < shi)) sn = Real(0.5) * (slo + shi);
                    if (m_abs(sn - s) <= Real(4) * RealLimits<Real>::eps() || shi - slo <= Real(4) * RealLimits<Real>::eps()) { s = sn; break; }
                    s = sn;
                }
                Real I, v;
                leg_tail<Real, G>(cR, s, &I, &v);
                IR += hw * I;
                ustar = mid + hw * s;
                found = true;
            } else {
                T += Ih[hh];
                Real sR = Real(0);
#pragma unroll
                for (int g = 0; g < G; g++) sR += GL<G>::template w<Real>(g) * vR[hh][g];
                IR += hw * sR;
            }
        }
        if (found) break;
        du = m_min(Real(1), Real(2) * (uk - ua));
        uk = ua;
    }
    if (!found) {
        // tail: T(u) = T + (ut - u)/Dinf + Rt(w), Rt(w) = int_w^wt (1/D - 1/Dinf)/w' dw'
        Real wte = m_exp(ut);
        Real cR0 = C.c * (Real(1) - xe) * (Real(1) - xe);
        Real qD[G], qR[G];
        const bool smooth = !clamped;
        Real iv[G], dvv[G];
        {
            auto node = [&](int l, Real &d) {
                d = d0 * (Real(0.5) * wte * (Real(1) + GL<G>::template x<Real>(l)));
                return Real(1) / ode_D<Real, NSMAX>(C, Q, xe, d);
            };
            ev.template eval<G>(node, iv, dvv);
        }
#pragma unroll
        for (int g = 0; g < G; g++) {
            Real w = Real(0.5) * wte * (Real(1) + GL<G>::template x<Real>(g));
            Real xi = xe + dvv[g];
            Real invD = iv[g];
            qD[g] = smooth ? (invD - Real(1) / Dinf) / w : Real(0);
            qR[g] = smooth ? (C.c * (Real(1) - xi) * (Real(1) - xi) * invD - cR0 / Dinf) / w : Real(0);
        }
        Real cD[G], cRc[G];
        leg_coeffs<Real, G>(qD, cD);
        leg_coeffs<Real, G>(qR, cRc);
        // Newton on T(u) = h: T(u) = T + (ut - u)/Dinf + Rt(e^u), dT/du = -1/D(u)
        // with 1/D = 1/Dinf + w q(w) from the interpolant; bracketed in [ulo, ut]
        Real u = ut - Dinf * (h - T);
        Real uhi = ut, ulo = -RealLimits<Real>::inf();
        for (int it = 0; it < 60; it++) {
            Real w = m_exp(u);
            Real s = Real(2) * w / wte - Real(1);
            if (s < Real(-1)) s = Real(-1);
            Real I, v;
            leg_tail<Real, G>(cD, s, &I, &v);
            Real g = T + (ut - u) / Dinf + Real(0.5) * wte * I - h;   // decreasing in u, g(ut) < 0
            if (g == Real(0)) break;
            if (g > Real(0)) ulo = u; else uhi = u;
            Real invD = Real(1) / Dinf + w * v;
            Real un = u + g / invD;
            if (!(un < uhi && un > ulo))
                un = (ulo > -RealLimits<Real>::inf()) ? Real(0.5) * (ulo + uhi) : u - (uhi - u) - Real(1);
            bool conv = m_abs(un - u) <= Real(8) * RealLimits<Real>::eps() * (Real(1) + m_abs(u));
            u = un;
            if (conv) break;
        }
        Real w = m_exp(u);
        Real s = Real(2) * w / wte - Real(1);
        if (s < Real(-1)) s = Real(-1);
        Real I, v;
        leg_tail<Real, G>(cRc, s, &I, &v);
        IR += cR0 * (ut - u) / Dinf + Real(0.5) * wte * I;
        ustar = u;
    }
    R.x = xe + d0 * m_exp(ustar);
    R.IR = IR;
    if (Eval::attenuation && C.b0 > Real(0))
        R.lnfav = attenuation_average<Real, NSMAX>(C, Q, xe, d0, Dinf, h, ustar, ut, found, wt);
    return R;
}


// Integrate one cell from x0 over h.  sigma0 scales the tabulated b (= n ds)
// to an optical depth for the curvature scale.
template <typename Real, int NSMAX = MAX_SRC>
OOTS_HD IntResult<Real> integrate_cell(const CellODE<Real> &C, Real x0, Real h, Real sigma0)
{
    IntResult<Real> R;
    Real F0, dF0, f0;
    if (integrate_prelude<Real, NSMAX>(C, x0, h, sigma0, R, F0, dF0, f0)) return R;
    return integrate_general<Real, NSMAX>(C, x0, h, sigma0, R, F0, dF0, f0, SeqEval());
}

// Second pass for A1 (Eq. 3): <exp(-b0 x)> over the step, once the end point
// u* is known.  Relative to the trajectory's smallest x the weight
// exp(-b0 (x - x_min)) is largest at that end and falls monotonically away
// from it, so the integral is marched from the heavy end with adaptive panels
// (relative to the sum so far) and stopped where the weight is negligible.
template <typename Real, int NSMAX>
OOTS_HD Real attenuation_average(const CellODE<Real> &C, const SrcEq<Real> *Q, Real xe, Real d0, Real Dinf,
                                 Real h, Real ustar, Real ut, bool in_panels, Real wt)
{
    constexpr int G = IntCfg<Real>::G;
    const Real xend = xe + d0 * m_exp(ustar);
    const Real xmin = m_min(xend, xe + d0);
    const Real wcut = Real(2) * IntCfg<Real>::umax();      // weight below e^-wcut is dropped
    Real S = Real(0), T2 = Real(0);   // weighted and unweighted time on the same nodes
    // tail part [u*, ut] (near-equilibrium: the weight varies by at most e^0.5 there)
    Real ustart = ustar;
    if (!in_panels) {
        const Real wte = m_exp(ut);
        const Real e0 = m_exp(-C.b0 * (xe - xmin));
        Real q[G], qt[G];
#pragma unroll
        for (int g = 0; g < G; g++) {
            Real w = Real(0.5) * wte * (Real(1) + GL<G>::template x<Real>(g));
            Real d = d0 * w;
            Real invD = Real(1) / ode_D<Real, NSMAX>(C, Q, xe, d);
            q[g] = (m_exp(-C.b0 * (xe + d - xmin)) * invD - e0 / Dinf) / w;
            qt[g] = (invD - Real(1) / Dinf) / w;
        }
        Real cq[G], cqt[G];
        leg_coeffs<Real, G>(q, cq);
        leg_coeffs<Real, G>(qt, cqt);
        Real s = Real(2) * m_exp(ustar) / wte - Real(1);
        if (s < Real(-1)) s = Real(-1);
        Real I, v;
        leg_tail<Real, G>(cq, s, &I, &v);
        S += e0 * (ut - ustar) / Dinf + Real(0.5) * wte * I;
        leg_tail<Real, G>(cqt, s, &I, &v);
        T2 += (ut - ustar) / Dinf + Real(0.5) * wte * I;
        ustart = ut;
    }
    // panel part [ustart, 0]: heavy end is u = ustart when x decreases (d0 > 0),
    // u = 0 when x increases (d0 < 0)
    const bool up = d0 > Real(0);          // march from ustart upward to 0
    Real pos = up ? ustart : Real(0);
    const Real end = up ? Real(0) : ustart;
    Real du = m_min(Real(1), Real(0.25) / m_max(C.b0 * m_abs(d0) * m_exp(pos), Real(1e-30)));
    int np = 0;
    while ((up ? pos < end : pos > end) && np < 600) {
        Real nxt = up ? m_min(pos + du, end) : m_max(pos - du, end);
        Real lo = m_min(pos, nxt), hi = m_max(pos, nxt);
        Real mid = Real(0.5) * (lo + hi), hw = Real(0.5) * (hi - lo);
        Real full = Real(0), halves = Real(0), thalves = Real(0);
#pragma unroll
        for (int g = 0; g < G; g++) {
            Real d = d0 * m_exp(mid + hw * GL<G>::template x<Real>(g));
            full += GL<G>::template w<Real>(g) * hw * m_exp(-C.b0 * (xe + d - xmin)) / ode_D<Real, NSMAX>(C, Q, xe, d);
        }
#pragma unroll
        for (int hh = 0; hh < 2; hh++) {
            Real m2 = mid + (hh ? Real(0.5) : Real(-0.5)) * hw;
#pragma unroll
            for (int g = 0; g < G; g++) {
                Real d = d0 * m_exp(m2 + Real(0.5) * hw * GL<G>::template x<Real>(g));
                Real invD = Real(1) / ode_D<Real, NSMAX>(C, Q, xe, d);
                halves += GL<G>::template w<Real>(g) * Real(0.5) * hw * m_exp(-C.b0 * (xe + d - xmin)) * invD;
                thalves += GL<G>::template w<Real>(g) * Real(0.5) * hw * invD;
            }
        }
        np++;
        if (m_abs(full - halves) > IntCfg<Real>::tolq() * Real(10) * (S + halves) && hw > Real(1e-12)) {
            du = hw;
            continue;
        }
        S += halves;
        T2 += thalves;
        pos = nxt;
        // once the weight is negligible, the rest only adds (unweighted) time
        Real xp = xe + d0 * m_exp(pos);
        if (C.b0 * (xp - xmin) > wcut) { T2 = h; break; }
        du = m_min(Real(1), Real(4) * hw);
    }
    Real fav = S / (T2 > Real(0) ? T2 : h);
    return -C.b0 * xmin + m_log(fav > Real(0) ? fav : RealLimits<Real>::eps());
}

// dx/dt at x
template <typename Real, int NSMAX = MAX_SRC>
OOTS_HD __forceinline__ Real ode_rhs(const CellODE<Real> &C, Real x)
{
    Real F, dF;
    ode_F<Real, NSMAX>(C, x, &F, &dF);
    return -F + C.c * (Real(1) - x) * (Real(1) - x);
}

} // namespace oots
