/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the on-the-spot (OTS) hydrogen
 * photoionisation hot path of Mackey (2012), "Accuracy and efficiency of
 * raytracing photoionisation algorithms" (arXiv:1201.5651).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product (the CUDA
 * library under paper_1201_5651_gb300/) never links, loads or calls it, and the
 * two share no code, headers, tables or constants.
 *
 * What it computes, in the paper's order and notation (x = neutral fraction =
 * 1 - y of the paper):
 *   - short-characteristics column densities from a vertex point source through
 *     a uniform Cartesian grid, octant by octant, cells visited in increasing
 *     i+j+k (Sect. 2: the raytracer, with the Mellema et al. 2006 weighting;
 *     Sect. 5: source moved to a cell vertex, octants traced independently);
 *   - the photon-conserving photoionisation rate per H atom of each cell
 *     (Sect. 2, Eq. 1-2: A_pi is a function of density, neutral fraction, the
 *     neutral column and the distance to the source);
 *   - the neutral-fraction ODE of Eq. 2 with T fixed and collisional ionisation
 *     off:  dx/dt = -F(x) + alpha_B n (1-x)^2, integrated with the column to the
 *     cell entry frozen and the cell's own optical depth evolving with x;
 *   - the timestep criteria of Eq. 4 (K1, K3, K4; K2 needs an energy equation);
 *   - the three schemes: A1 implicit (Sect. 2.1, Eq. 3), A2 first-order explicit
 *     and A3 second-order explicit (Sect. 2.2, Fig. 1);
 *   - frequency-integrated rate tables for a blackbody source (Sect. 2, the
 *     paragraph on multi-frequency rates; Sect. 4);
 *   - brute-force long characteristics (exact voxel traversal), used only to
 *     bound the accuracy of the short characteristics;
 *   - plane-parallel sources (a source at infinity whose rays run parallel to
 *     a grid axis, the slab test of Sect. 3.1): the column to a cell is the sum
 *     of n x dx of the cells before it on its row, and the rate of a cell is
 *     the photon flux it removes per unit face area over n dx.
 *
 * Readings where the paper is silent (each is a parameter or a stated choice):
 *   - rate form: absorbed photons per atom per second
 *       F = [R_in - R_out(x)] / (n V_sh),  V_sh = 4 pi r^2 ds,
 *     r = distance from the source vertex to the cell centre, ds = chord of the
 *     central ray through the cell;
 *   - SC weights: bilinear weights of the entry point on the upwind layer of
 *     the dominant axis, divided by max(dtau_nb, tau0), normalised; ties of the
 *     dominant axis are averaged over the tied axes; out-of-octant neighbours
 *     are dropped;
 *   - integrator: the exact solution of the scalar autonomous ODE, obtained
 *     here by an adaptive Dormand-Prince 5(4) integration in the variable
 *     u = ln((x - x_eq)/(x0 - x_eq)), where x_eq is the unique root of the
 *     right-hand side (it is strictly decreasing in x);
 *   - tables: ln(P/Q) on log-spaced columns, interpolated by the quintic
 *     Hermite polynomial in ln N through the node values and the exact first
 *     and second logarithmic derivatives; below the first node P is linear in
 *     N; above the last node P = 0; sigma_nu = sigma0 (nu/nu0)^-3; blackbody
 *     photon spectrum nu^2/(exp(h nu/kT) - 1) on [nu0, numax].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define OR_PI 3.14159265358979323846

/* Threshold photon energy h nu0 = 13.6 eV (Sect. 2.1) over Boltzmann's
 * constant in eV/K: theta = h nu0 / (k T) = OR_TNU0 / T. */
#define OR_TNU0 (13.6 / 8.617333262e-5)

/* ------------------------------------------------------------------------ */
/* Problem description                                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;        /* cells per axis; index = X + nx*(Y + ny*Z)        */
    double dx;             /* cell side [cm]                                   */
    double alpha;          /* case-B recombination coefficient [cm^3 s^-1]     */
    double sigma0;         /* threshold photoionisation cross-section [cm^2]   */
    double tau0;           /* optical-depth floor of the SC weights            */
    const double *nH;      /* hydrogen number density per cell [cm^-3]         */
    int nsrc;              /* number of point sources                          */
    const int *vtx;        /* 3 per source: vertex indices (0..n)              */
    const double *Q;       /* ionising photon rate per source [s^-1]           */
    const int *kind;       /* per source: 0 monochromatic, 1 tabulated         */
    const double *tabL;    /* per source, K values: ln(P/Q) at the nodes       */
    const double *tabD1;   /* per source, K values: d ln P / d ln N            */
    const double *tabD2;   /* per source, K values: d2 ln P / d (ln N)^2       */
    int K;                 /* table nodes                                      */
    double lnN_lo, lnN_hi; /* ln of the first and last node column [cm^-2]     */
    const int *plane;      /* per source (NULL: all point sources): -1 for a
                              vertex point source; 2*axis + back for a plane
                              source whose rays run along +axis (back = 0) or
                              -axis (back = 1).  A plane source's Q is its
                              photon flux F_gamma [cm^-2 s^-1].                */
} or_problem;

typedef struct {
    int scheme;            /* 1 = A1 implicit, 2 = A2, 3 = A3                  */
    double K1, K3, K4;     /* Eq. 4 factors; <= 0 means "not used"             */
    double dt_fixed;       /* > 0: fixed timestep (still capped at t_end - t)  */
} or_scheme;

/* ------------------------------------------------------------------------ */
/* Rate tables (frequency-integrated photon rate through a column N)         */
/* ------------------------------------------------------------------------ */

/* Photon spectrum (per unit x = nu/nu0) and cross-section. */
static double bb_phi(double xnu, double theta) { return xnu * xnu / expm1(theta * xnu); }

typedef struct { double theta, sigma0, N; int moment; double mu; } bb_args;

/* Integrand of the m-th moment: phi * sigma^m * exp(-sigma N), with the
 * "centred" second moment phi (sigma - mu)^2 exp(-sigma N) for m = 3 and the
 * deficit phi * (exp(-sigma N) - 1) for m = 4. */
static double bb_integrand(double xnu, const bb_args *a)
{
    double s = a->sigma0 / (xnu * xnu * xnu);
    if (a->moment == 4) return bb_phi(xnu, a->theta) * expm1(-s * a->N);
    double w = bb_phi(xnu, a->theta) * exp(-s * a->N);
    switch (a->moment) {
    case 0: return w;
    case 1: return w * s;
    default: return w * (s - a->mu) * (s - a->mu);
    }
}

/* Adaptive Gauss-Kronrod 7-15 on [lo, hi], recursive bisection. */
static const double gk_x[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.0};
static const double gk_wk[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = { /* Gauss weights at gk_x[1], [3], [5], [7] */
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static double gk_rec(const bb_args *a, double lo, double hi, double tol, int depth)
{
    double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
    double k = 0.0, g = 0.0;
    for (int i = 0; i < 8; i++) {
        double f1 = bb_integrand(c - h * gk_x[i], a);
        double f2 = (i == 7) ? 0.0 : bb_integrand(c + h * gk_x[i], a);
        double fs = f1 + f2;
        k += gk_wk[i] * fs;
        if (i & 1) g += gk_wg[i >> 1] * fs;
    }
    k *= h; g *= h;
    if (fabs(k - g) <= tol || fabs(k - g) <= 1e-11 * fabs(k) || depth > 30)
        return k;
    return gk_rec(a, lo, c, 0.5 * tol, depth + 1) + gk_rec(a, c, hi, 0.5 * tol, depth + 1);
}

static double bb_moment(const bb_args *a, double xlo, double xhi, double scale)
{
    /* split into a few panels so the recursion starts from a sensible grid */
    double sum = 0.0;
    int np = 16;
    double r = pow(xhi / xlo, 1.0 / np);
    double lo = xlo;
    for (int i = 0; i < np; i++) {
        double hi = (i == np - 1) ? xhi : lo * r;
        sum += gk_rec(a, lo, hi, 1e-13 * scale / np, 0);
        lo = hi;
    }
    return sum;
}

/*
 * Build the table of a source spectrum on K log-spaced columns
 * N_k = exp(lnN_lo + k (lnN_hi - lnN_lo)/(K-1)):
 *   L[k]  = ln(P(N_k)/Q),   P(N) = Q * int phi e^{-sigma N} / int phi
 *   D1[k] = d ln P / d ln N = -N <sigma>
 *   D2[k] = d2 ln P / d(ln N)^2 = -N <sigma> + N^2 var(sigma)
 * where <.> and var are weighted by phi e^{-sigma N}.
 * kind 0: a delta spectrum at nu0 (P = Q e^{-sigma0 N}, exact);
 * kind 1: blackbody of temperature Tbb on [nu0, numax_over_nu0 nu0].
 */
int or_table_build(int kind, double Tbb, double sigma0, double numax_over_nu0,
                   int K, double lnN_lo, double lnN_hi,
                   double *L, double *D1, double *D2)
{
    if (K < 2 || !(lnN_hi > lnN_lo)) return -1;
    double dl = (lnN_hi - lnN_lo) / (K - 1);
    if (kind == 0) {
        for (int k = 0; k < K; k++) {
            double N = exp(lnN_lo + k * dl);
            L[k] = -sigma0 * N;
            D1[k] = -sigma0 * N;
            D2[k] = -sigma0 * N;
        }
        return 0;
    }
    if (kind != 1 || !(Tbb > 0) || !(numax_over_nu0 > 1)) return -1;
    bb_args a;
    a.theta = OR_TNU0 / Tbb;
    a.sigma0 = sigma0;
    a.N = 0.0; a.moment = 0; a.mu = 0.0;
    double Z = bb_moment(&a, 1.0, numax_over_nu0, 1.0);
    Z = bb_moment(&a, 1.0, numax_over_nu0, Z);
    Z = bb_moment(&a, 1.0, numax_over_nu0, Z);
    for (int k = 0; k < K; k++) {
        double N = exp(lnN_lo + k * dl);
        a.N = N;
        a.moment = 0;
        double m0 = bb_moment(&a, 1.0, numax_over_nu0, Z);
        m0 = bb_moment(&a, 1.0, numax_over_nu0, m0);
        m0 = bb_moment(&a, 1.0, numax_over_nu0, m0);
        a.moment = 1;
        double m1 = bb_moment(&a, 1.0, numax_over_nu0, m0 * sigma0);
        double mu = m1 / m0;
        a.moment = 3; a.mu = mu;
        double v = bb_moment(&a, 1.0, numax_over_nu0, m0 * mu * mu) / m0;
        if (m0 > 0.5 * Z) {
            /* thin columns: ln(P/Q) = log1p(int phi (e^{-sigma N} - 1) / Z), no cancellation */
            a.moment = 4;
            double def = bb_moment(&a, 1.0, numax_over_nu0, Z - m0);
            def = bb_moment(&a, 1.0, numax_over_nu0, fabs(def) > 0 ? fabs(def) : 1e-300);
            L[k] = log1p(def / Z);
        } else {
            L[k] = log(m0 / Z);
        }
        D1[k] = -N * mu;
        D2[k] = -N * mu + N * N * v;
    }
    return 0;
}

/* Quintic Hermite basis on t in [0,1] and the derivative of the interpolant. */
static double herm5(const double *y, double t, double dl)
{
    /* y: value0, d1_0, d2_0, value1, d1_1, d2_1 in ln N units; dl = node step */
    double t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
    double h0 = 1 - 10 * t3 + 15 * t4 - 6 * t5;
    double h1 = t - 6 * t3 + 8 * t4 - 3 * t5;
    double h2 = 0.5 * (t2 - 3 * t3 + 3 * t4 - t5);
    double h3 = 0.5 * (t3 - 2 * t4 + t5);
    double h4 = -4 * t3 + 7 * t4 - 3 * t5;
    double h5 = 10 * t3 - 15 * t4 + 6 * t5;
    return y[0] * h0 + y[1] * dl * h1 + y[2] * dl * dl * h2
         + y[5] * dl * dl * h3 + y[4] * dl * h4 + y[3] * h5;
}

/* d/dlambda of the interpolant (lambda = ln N), at local t. */
static double herm5_deriv(const double *y, double t, double dl)
{
    double t2 = t * t, t3 = t2 * t, t4 = t3 * t;
    double d0 = -30 * t2 + 60 * t3 - 30 * t4;
    double d1 = 1 - 18 * t2 + 32 * t3 - 15 * t4;
    double d2 = 0.5 * (2 * t - 9 * t2 + 12 * t3 - 5 * t4);
    double d3 = 0.5 * (3 * t2 - 8 * t3 + 5 * t4);
    double d4 = -12 * t2 + 28 * t3 - 15 * t4;
    double d5 = 30 * t2 - 60 * t3 + 30 * t4;
    return (y[0] * d0 + y[1] * dl * d1 + y[2] * dl * dl * d2
          + y[5] * dl * dl * d3 + y[4] * dl * d4 + y[3] * d5) / dl;
}

typedef struct { const double *L, *D1, *D2; int K; double lnN_lo, lnN_hi; } or_tab;

static void tab_node(const or_tab *T, int k, double *y)
{
    y[0] = T->L[k]; y[1] = T->D1[k]; y[2] = T->D2[k];
    y[3] = T->L[k + 1]; y[4] = T->D1[k + 1]; y[5] = T->D2[k + 1];
}

/* ln(P(N)/Q); -inf above the table. */
double or_tab_lnp(const or_tab *T, double N)
{
    double dl = (T->lnN_hi - T->lnN_lo) / (T->K - 1);
    double N0 = exp(T->lnN_lo);
    if (N <= 0.0) return 0.0;
    if (N < N0) return log1p(expm1(T->L[0]) * (N / N0));
    double lam = log(N);
    if (lam > T->lnN_hi) return -INFINITY;
    int k = (int)floor((lam - T->lnN_lo) / dl);
    if (k > T->K - 2) k = T->K - 2;
    if (k < 0) k = 0;
    double y[6];
    tab_node(T, k, y);
    return herm5(y, (lam - (T->lnN_lo + k * dl)) / dl, dl);
}

/*
 * ln P(Na + dN) - ln P(Na) for dN >= 0, without cancellation: below the table
 * from the closed form of the linear piece, inside the table as the integral
 * of the interpolant's derivative over each node interval (3-point
 * Gauss-Legendre, exact for the quartic derivative), the length of each
 * piece in ln N taken from log1p of the relative column increment.
 */
double or_tab_dlnp(const or_tab *T, double Na, double dN)
{
    if (dN <= 0.0) return 0.0;
    double dl = (T->lnN_hi - T->lnN_lo) / (T->K - 1);
    double N0 = exp(T->lnN_lo), Nhi = exp(T->lnN_hi);
    if (Na + dN > Nhi) return -INFINITY;
    double acc = 0.0;
    double lo = Na;       /* start of the current piece          */
    double rem = dN;      /* column still to cover (kept exactly) */
    if (lo < N0) {
        double piece = (N0 - lo) < rem ? (N0 - lo) : rem;
        double a = -expm1(T->L[0]);           /* 1 - P(N0)/Q */
        acc += log1p(-a * piece / (N0 - a * lo));
        if (piece >= rem) return acc;
        lo = N0;
        rem -= piece;
    }
    static const double gx[3] = {-0.774596669241483377035853079956480, 0.0,
                                 0.774596669241483377035853079956480};
    static const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
    /* integral of the interpolant's derivative over [lo, lo + piece] inside interval k */
#define OR_PIECE(k_, lo_, piece_)                                                      \
    do {                                                                               \
        double len_ = log1p((piece_) / (lo_));                                         \
        double lam_ = log(lo_), lam0_ = T->lnN_lo + (k_) * dl, y_[6], sum_ = 0.0;      \
        tab_node(T, (k_), y_);                                                         \
        for (int g = 0; g < 3; g++)                                                    \
            sum_ += gw[g] * herm5_deriv(y_, (lam_ + 0.5 * len_ * (1.0 + gx[g]) - lam0_) / dl, dl); \
        acc += 0.5 * len_ * sum_;                                                      \
    } while (0)
    int k = (int)floor((log(lo) - T->lnN_lo) / dl);
    if (k > T->K - 2) k = T->K - 2;
    if (k < 0) k = 0;
    double Nk1 = exp(T->lnN_lo + (k + 1) * dl);
    if (Nk1 <= lo && k < T->K - 2) { k++; Nk1 = exp(T->lnN_lo + (k + 1) * dl); }
    if (rem <= Nk1 - lo) {                  /* the step stays inside one interval */
        OR_PIECE(k, lo, rem);
        return acc;
    }
    OR_PIECE(k, lo, Nk1 - lo);              /* first partial interval */
    rem -= Nk1 - lo;
    double Nend = Nk1 + rem;
    int k2 = (int)floor((log(Nend) - T->lnN_lo) / dl);
    if (k2 > T->K - 2) k2 = T->K - 2;
    if (k2 < k + 1) k2 = k + 1;
    double Nk2 = exp(T->lnN_lo + k2 * dl);
    if (Nk2 > Nend && k2 > k + 1) { k2--; Nk2 = exp(T->lnN_lo + k2 * dl); }
    acc += T->L[k2] - T->L[k + 1];          /* whole intervals: node differences */
    double last = (k2 == k + 1) ? rem : Nend - Nk2;
    if (last > 0.0) OR_PIECE(k2, Nk2, last); /* last partial interval */
#undef OR_PIECE
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

/* Octant-local index of global cell index X along an axis whose source
 * vertex is v (the octant side is chosen by X >= v). */
static int oct_local(int X, int v) { return X >= v ? X - v : v - 1 - X; }

/* Cell geometry relative to a vertex source, in units of dx:
 * c = (i+1/2, j+1/2, k+1/2); r2 = |c|^2; sfac = |c| / max(c) = ds/dx. */
static void cell_geom(const or_problem *p, int s, int X, int Y, int Z,
                      int *ijk, double *r2, double *sfac)
{
    const int *v = p->vtx + 3 * s;
    ijk[0] = oct_local(X, v[0]);
    ijk[1] = oct_local(Y, v[1]);
    ijk[2] = oct_local(Z, v[2]);
    double c0 = ijk[0] + 0.5, c1 = ijk[1] + 0.5, c2 = ijk[2] + 0.5;
    double cm = c0 > c1 ? c0 : c1;
    cm = cm > c2 ? cm : c2;
    *r2 = c0 * c0 + c1 * c1 + c2 * c2;
    *sfac = sqrt(*r2) / cm;
}

/* -1 for a vertex point source, else the plane code 2*axis + back. */
static int src_plane(const or_problem *p, int s) { return p->plane ? p->plane[s] : -1; }

/* Ray segment ds through the cell (X,Y,Z) and the volume V_sh over which the
 * photons it removes are shared, for source s:
 *   point source: ds = dx |c|/max(c), V_sh = 4 pi r^2 ds (per unit Q);
 *   plane source: ds = dx and V_sh = dx, the cell volume per unit face area
 *                 (Q is then a flux per unit area). */
static void src_shell(const or_problem *p, int s, int X, int Y, int Z, double *ds, double *Vsh)
{
    if (src_plane(p, s) >= 0) {
        *ds = p->dx;
        *Vsh = p->dx;
        return;
    }
    int ijk[3]; double r2, sf;
    cell_geom(p, s, X, Y, Z, ijk, &r2, &sf);
    *ds = p->dx * sf;
    *Vsh = 4.0 * OR_PI * r2 * p->dx * p->dx * *ds;
}

/* Photons per second source s emits into the grid: Q for a point source; for
 * a plane source its flux times the area of the face it enters through. */
static double src_emission(const or_problem *p, int s)
{
    int code = src_plane(p, s);
    if (code < 0) return p->Q[s];
    int n3[3] = {p->nx, p->ny, p->nz};
    int axis = code / 2;
    return p->Q[s] * (double)n3[(axis + 1) % 3] * (double)n3[(axis + 2) % 3] * p->dx * p->dx;
}

/* Cell (u, w) of row m, counted along the direction of travel of plane code
 * `code`: u and w index the two transverse axes (axis+1, axis+2 mod 3). */
static long plane_cell(const or_problem *p, int code, int m, int u, int w)
{
    int axis = code / 2, back = code & 1;
    int n3[3] = {p->nx, p->ny, p->nz};
    int G[3];
    G[axis] = back ? n3[axis] - 1 - m : m;
    G[(axis + 1) % 3] = u;
    G[(axis + 2) % 3] = w;
    return G[0] + (long)p->nx * (G[1] + (long)p->ny * G[2]);
}

/* ------------------------------------------------------------------------ */
/* Short-characteristics trace                                               */
/* ------------------------------------------------------------------------ */

/*
 * Interpolated column to the entry of cell (i,j,k) of one octant, from the
 * N_out and dtau of its upwind neighbours (full-grid arrays).
 */
static double sc_interp(const or_problem *p, const int *v, const int *sg, const int *ext,
                        int i, int j, int k, const double *Nout, const double *dtau)
{
    int idx[3] = {i, j, k};
    int c2[3] = {2 * i + 1, 2 * j + 1, 2 * k + 1};   /* twice the centre coordinates */
    int cm = c2[0];
    if (c2[1] > cm) cm = c2[1];
    if (c2[2] > cm) cm = c2[2];
    double sum = 0.0;
    int ntied = 0;
    for (int a = 0; a < 3; a++) {
        if (c2[a] != cm) continue;
        ntied++;
        if (idx[a] == 0) continue;            /* only the cell at the vertex */
        int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
        double d1 = (double)c2[t1] / (double)c2[a];  /* weight of the t-1 neighbour */
        double d2 = (double)c2[t2] / (double)c2[a];
        double ws = 0.0, wn = 0.0;
        for (int e1 = 0; e1 < 2; e1++) {
            for (int e2 = 0; e2 < 2; e2++) {
                int nb[3];
                nb[a] = idx[a] - 1;
                nb[t1] = idx[t1] - e1;
                nb[t2] = idx[t2] - e2;
                if (nb[t1] < 0 || nb[t2] < 0) continue;   /* outside the octant */
                (void)ext;
                int G[3];
                for (int q = 0; q < 3; q++) G[q] = sg[q] > 0 ? v[q] + nb[q] : v[q] - 1 - nb[q];
                long gi = G[0] + (long)p->nx * (G[1] + (long)p->ny * G[2]);
                double wg = (e1 ? d1 : 1.0 - d1) * (e2 ? d2 : 1.0 - d2);
                double dt = dtau[gi] > p->tau0 ? dtau[gi] : p->tau0;
                double w = wg / dt;
                ws += w;
                wn += w * Nout[gi];
            }
        }
        sum += wn / ws;
    }
    return sum / ntied;
}

/*
 * Column density of neutral hydrogen to the entry of every cell, for source s,
 * from the neutral fractions x.  Nin[cell] receives N_in; if dtau_out is not
 * NULL it receives the cell optical depth sigma0 n x ds used by the weights.
 */
void or_trace(const or_problem *p, int s, const double *x, double *Nin, double *dtau_out)
{
    long ncell = (long)p->nx * p->ny * p->nz;
    int code = src_plane(p, s);
    if (code >= 0) {
        /* rays parallel to the axis: each row is traced from the face the
         * photons enter through, with no interpolation */
        int n3[3] = {p->nx, p->ny, p->nz};
        int axis = code / 2;
        for (int w = 0; w < n3[(axis + 2) % 3]; w++)
            for (int u = 0; u < n3[(axis + 1) % 3]; u++) {
                double N = 0.0;
                for (int m = 0; m < n3[axis]; m++) {
                    long gi = plane_cell(p, code, m, u, w);
                    double dN = p->nH[gi] * x[gi] * p->dx;
                    Nin[gi] = N;
                    if (dtau_out) dtau_out[gi] = p->sigma0 * dN;
                    N += dN;
                }
            }
        return;
    }
    double *Nout = (double *)malloc(sizeof(double) * ncell);
    double *dtau = dtau_out ? dtau_out : (double *)malloc(sizeof(double) * ncell);
    const int *v = p->vtx + 3 * s;
    int n3[3] = {p->nx, p->ny, p->nz};
    for (int oct = 0; oct < 8; oct++) {
        int sg[3] = {(oct & 1) ? -1 : 1, (oct & 2) ? -1 : 1, (oct & 4) ? -1 : 1};
        int ext[3];
        for (int q = 0; q < 3; q++) ext[q] = sg[q] > 0 ? n3[q] - v[q] : v[q];
        if (ext[0] <= 0 || ext[1] <= 0 || ext[2] <= 0) continue;
        int mmax = ext[0] + ext[1] + ext[2] - 3;
        for (int m = 0; m <= mmax; m++) {
            for (int i = 0; i < ext[0] && i <= m; i++) {
                for (int j = 0; j < ext[1] && i + j <= m; j++) {
                    int k = m - i - j;
                    if (k >= ext[2]) continue;
                    int G[3] = {sg[0] > 0 ? v[0] + i : v[0] - 1 - i,
                                sg[1] > 0 ? v[1] + j : v[1] - 1 - j,
                                sg[2] > 0 ? v[2] + k : v[2] - 1 - k};
                    long gi = G[0] + (long)p->nx * (G[1] + (long)p->ny * G[2]);
                    double nin = (m == 0) ? 0.0 : sc_interp(p, v, sg, ext, i, j, k, Nout, dtau);
                    double c0 = i + 0.5, c1 = j + 0.5, c2 = k + 0.5;
                    double cm = c0 > c1 ? c0 : c1;
                    cm = cm > c2 ? cm : c2;
                    double ds = p->dx * sqrt(c0 * c0 + c1 * c1 + c2 * c2) / cm;
                    double dN = p->nH[gi] * x[gi] * ds;
                    Nin[gi] = nin;
                    Nout[gi] = nin + dN;
                    dtau[gi] = p->sigma0 * dN;
                }
            }
        }
    }
    free(Nout);
    if (!dtau_out) free(dtau);
}

/* ------------------------------------------------------------------------ */
/* Per-cell rates and the neutral-fraction ODE                               */
/* ------------------------------------------------------------------------ */

/* Rate parameters of one source for one cell.
 *   monochromatic: F(x) = A (1 - exp(-b x)),  A = Q e^{-sigma0 Nin}/(n V_sh),
 *                  b = sigma0 n ds;
 *   tabulated:     F(x) = A [P(Nin) - P(Nin + b x)]/Q, A = Q/(n V_sh), b = n ds. */
typedef struct { int kind; double A, b, Nin; or_tab tab; } or_srcrate;

typedef struct {
    int ns;
    const or_srcrate *r;
    double c;     /* alpha n */
    double b0;    /* sigma0 n ds of the attenuation integrated by A1 */
} or_cell;

static double src_F(const or_srcrate *r, double x)
{
    if (r->A == 0.0) return 0.0;
    if (r->kind == 0) return r->A * (-expm1(-r->b * x));
    double lp = or_tab_lnp(&r->tab, r->Nin);
    if (lp == -INFINITY) return 0.0;
    return r->A * exp(lp) * (-expm1(or_tab_dlnp(&r->tab, r->Nin, r->b * x)));
}

/* F_s(xe + d) - F_s(xe), computed without cancellation. */
static double src_dF(const or_srcrate *r, double xe, double d)
{
    if (r->A == 0.0 || d == 0.0) return 0.0;
    if (r->kind == 0) {
        /* A (e^{-b xe} - e^{-b (xe + d)}), written so that no factor exceeds 1 */
        if (d > 0) return r->A * exp(-r->b * xe) * (-expm1(-r->b * d));
        return -r->A * exp(-r->b * (xe + d)) * (-expm1(r->b * d));
    }
    double Ne = r->Nin + r->b * xe;
    if (d > 0) {
        double lp = or_tab_lnp(&r->tab, Ne);
        if (lp == -INFINITY) return 0.0;
        return r->A * exp(lp) * (-expm1(or_tab_dlnp(&r->tab, Ne, r->b * d)));
    } else {
        double Nl = r->Nin + r->b * (xe + d);
        double lp = or_tab_lnp(&r->tab, Nl);
        if (lp == -INFINITY) return 0.0;
        return -r->A * exp(lp) * (-expm1(or_tab_dlnp(&r->tab, Nl, -r->b * d)));
    }
}

static double cell_F(const or_cell *C, double x)
{
    double s = 0.0;
    for (int i = 0; i < C->ns; i++) s += src_F(&C->r[i], x);
    return s;
}

static double cell_f(const or_cell *C, double x)
{
    return -cell_F(C, x) + C->c * (1.0 - x) * (1.0 - x);
}

/* Secant slope D = -(f(xe+d) - f(xe))/d > 0 of the right-hand side about its
 * root xe, in a form free of cancellation for small |d|. */
static double cell_D(const or_cell *C, double xe, double d)
{
    double s = 0.0;
    if (d == 0.0) {
        /* limit d -> 0: -f'(xe) */
        for (int i = 0; i < C->ns; i++) {
            const or_srcrate *r = &C->r[i];
            if (r->A == 0.0) continue;
            if (r->kind == 0) s += r->A * r->b * exp(-r->b * xe);
            else {
                /* F'(x) = A b P(Nin + b x) sigma_eff / Q with
                 * sigma_eff = -(d ln P/d ln N)/N at N = Nin + b xe */
                double Ne = r->Nin + r->b * xe;
                double lp = or_tab_lnp(&r->tab, Ne);
                if (lp == -INFINITY) continue;
                /* derivative of ln P by a tiny one-sided difference quotient of
                 * the exact stable difference */
                double dN = 1e-9 * (Ne > 1.0 ? Ne : 1.0);
                double g = or_tab_dlnp(&r->tab, Ne, dN) / dN;   /* d ln P / dN */
                s += -r->A * r->b * exp(lp) * g;
            }
        }
        return s + 2.0 * C->c * (1.0 - xe);
    }
    if (fabs(d) < 1e-250) return cell_D(C, xe, 0.0);   /* the limit, before anything underflows */
    for (int i = 0; i < C->ns; i++) {
        const or_srcrate *r = &C->r[i];
        if (r->A == 0.0) continue;
        if (r->kind == 0) {
            /* (F(xe + d) - F(xe))/d = A b e^{-b xe} (1 - e^{-z})/z, z = b d: the ratio
             * is formed before the products so that it cannot underflow */
            double z = r->b * d;
            if (z > -20.0) {
                double q = (z != 0.0) ? -expm1(-z) / z : 1.0;
                s += r->A * r->b * exp(-r->b * xe) * q;
            } else {
                /* far below the root: the two transmitted fractions directly */
                s += r->A * (exp(-r->b * xe) - exp(-r->b * (xe + d))) / d;
            }
        } else {
            s += src_dF(r, xe, d) / d;
        }
    }
    return s + C->c * (2.0 * (1.0 - xe) - d);
}

/* Root of the (strictly decreasing) right-hand side on [0,1] by bisection. */
static double cell_xeq(const or_cell *C, double x0, double f0)
{
    double lo, hi;
    if (f0 < 0) { lo = 0.0; hi = x0; }
    else { lo = x0; hi = 1.0; }
    double flo = cell_f(C, lo), fhi = cell_f(C, hi);
    if (flo <= 0.0) return lo;
    if (fhi >= 0.0) return hi;
    for (int it = 0; it < 2000; it++) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double fm = cell_f(C, mid);
        if (fm > 0) lo = mid;
        else if (fm < 0) hi = mid;
        else return mid;
    }
    /* pick the end with the smaller residual */
    return fabs(cell_f(C, lo)) <= fabs(cell_f(C, hi)) ? lo : hi;
}

/* Result of one cell integration over h. */
typedef struct {
    double x;       /* x(h)                                                  */
    double IF;      /* int_0^h F(x(t)) dt: photons absorbed per H atom       */
    double IR;      /* int_0^h alpha n (1-x)^2 dt: recombinations per atom   */
    double lnfav;   /* ln( (1/h) int_0^h exp(-b0 x(t)) dt )                  */
} or_intres;

/* Right-hand side of the system in normalised time s = t/h:
 *   y = (u, IF, IR, J),  xi = xe + d0 e^u,
 *   du/ds = -h D,  dIF/ds = h F(xi),  dIR/ds = h c (1-xi)^2,
 *   dJ/ds = exp(-b0 (xi - xref))                                            */
static void int_rhs(const or_cell *C, double xe, double d0, double h, double xref,
                    const double *y, double *dy)
{
    double d = d0 * exp(y[0]);
    double xi = xe + d;
    dy[0] = -h * cell_D(C, xe, d);
    dy[1] = h * cell_F(C, xi);
    dy[2] = h * C->c * (1.0 - xi) * (1.0 - xi);
    dy[3] = exp(-C->b0 * (xi - xref));
}

/* Dormand-Prince 5(4) tableau. */
static const double dp_a[7][6] = {
    {0},
    {1.0 / 5},
    {3.0 / 40, 9.0 / 40},
    {44.0 / 45, -56.0 / 15, 32.0 / 9},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
static const double dp_b5[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0};
static const double dp_b4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                                -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

/*
 * Exact solution (to ~1e-13) of dx/dt = f(x) = -F(x) + c (1-x)^2 over h, with
 * the time integrals of F, of the recombination term and of exp(-b0 x).
 */
/* One Dormand-Prince pass over [0, h]; xref is the reference point of the
 * attenuation integrand (the smallest x on the trajectory keeps it <= 1). */
static void dp_pass(const or_cell *C, double xe, double d0, double h, double xref, double *y)
{
    y[0] = y[1] = y[2] = y[3] = 0.0;
    double s = 0.0, ds = 1e-3;
    double D0 = cell_D(C, xe, d0);
    if (h * D0 > 0) ds = fmin(1.0, 0.05 / (h * D0));
    const double rtol = 1e-13, atol = 1e-14;
    double k[7][4], yt[4], y5[4];
    int nstep = 0;
    while (s < 1.0 && nstep < 2000000) {
        if (ds > 1.0 - s) ds = 1.0 - s;
        int_rhs(C, xe, d0, h, xref, y, k[0]);
        for (int st = 1; st < 7; st++) {
            for (int q = 0; q < 4; q++) {
                double acc = y[q];
                for (int j = 0; j < st; j++) acc += ds * dp_a[st][j] * k[j][q];
                yt[q] = acc;
            }
            int_rhs(C, xe, d0, h, xref, yt, k[st]);
        }
        double err = 0.0;
        for (int q = 0; q < 4; q++) {
            double a5 = y[q], a4 = y[q];
            for (int j = 0; j < 7; j++) { a5 += ds * dp_b5[j] * k[j][q]; a4 += ds * dp_b4[j] * k[j][q]; }
            y5[q] = a5;
            double sc = atol + rtol * fmax(fabs(y[q]), fabs(a5));
            double r = fabs(a5 - a4) / sc;
            if (r > err) err = r;
        }
        nstep++;
        if (err <= 1.0) {
            s += ds;
            memcpy(y, y5, 4 * sizeof(double));
            /* e^u underflowed: the state is the root itself from here on */
            if (d0 * exp(y[0]) == 0.0) {
                double rem = 1.0 - s;
                y[1] += h * rem * cell_F(C, xe);
                y[2] += h * rem * C->c * (1 - xe) * (1 - xe);
                y[3] += rem * exp(-C->b0 * (xe - xref));
                break;
            }
        }
        double fac = err > 0 ? 0.9 * pow(err, -0.2) : 5.0;
        if (fac > 5.0) fac = 5.0;
        if (fac < 0.2) fac = 0.2;
        ds *= fac;
    }
}

/*
 * Exact solution (to ~1e-13) of dx/dt = f(x) = -F(x) + c (1-x)^2 over h, with
 * the time integrals of F, of the recombination term and of exp(-b0 x).
 * The trajectory is monotone between x0 and x_eq, so its smallest x is
 * min(x0, x(h)); the attenuation is integrated relative to that point in a
 * second pass, once x(h) is known, so that it never underflows.
 */
or_intres or_integrate_cell(const or_cell *C, double x0, double h)
{
    or_intres R;
    R.x = x0; R.IF = 0; R.IR = 0; R.lnfav = -C->b0 * x0;
    if (!(h > 0)) return R;
    double f0 = cell_f(C, x0);
    double xe = (f0 == 0.0) ? x0 : cell_xeq(C, x0, f0);
    double d0 = x0 - xe;
    if (d0 == 0.0) {
        R.IF = h * cell_F(C, x0);
        R.IR = h * C->c * (1 - x0) * (1 - x0);
        return R;
    }
    double y[4];
    dp_pass(C, xe, d0, h, x0 < xe ? x0 : xe, y);
    R.x = xe + d0 * exp(y[0]);
    R.IF = y[1];
    R.IR = y[2];
    if (C->b0 > 0) {
        double xref = x0 < R.x ? x0 : R.x;
        dp_pass(C, xe, d0, h, xref, y);
        R.lnfav = -C->b0 * xref + log(y[3]);
    } else {
        R.lnfav = 0.0;
    }
    return R;
}

/* Flat-argument entry point for tests of the integrator alone.
 * kind/A/b/Nin: ns entries; tables (if any kind == 1) taken from p for the
 * source index in tabsrc[i].  out: x, IF, IR, lnfav. */
void or_integrate(int ns, const int *kind, const double *A, const double *b, const double *Nin,
                  const int *tabsrc, const or_problem *p, double c, double b0,
                  double x0, double h, double *out)
{
    or_srcrate r[64];
    if (ns > 64) ns = 64;
    for (int i = 0; i < ns; i++) {
        r[i].kind = kind[i]; r[i].A = A[i]; r[i].b = b[i]; r[i].Nin = Nin[i];
        if (kind[i] == 1) {
            int s = tabsrc[i];
            r[i].tab.L = p->tabL + (long)s * p->K;
            r[i].tab.D1 = p->tabD1 + (long)s * p->K;
            r[i].tab.D2 = p->tabD2 + (long)s * p->K;
            r[i].tab.K = p->K; r[i].tab.lnN_lo = p->lnN_lo; r[i].tab.lnN_hi = p->lnN_hi;
        }
    }
    or_cell C = {ns, r, c, b0};
    or_intres R = or_integrate_cell(&C, x0, h);
    out[0] = R.x; out[1] = R.IF; out[2] = R.IR; out[3] = R.lnfav;
}

/* Table evaluation entry points for tests (source s of problem p). */
double or_lnp(const or_problem *p, int s, double N)
{
    or_tab T = {p->tabL + (long)s * p->K, p->tabD1 + (long)s * p->K, p->tabD2 + (long)s * p->K,
                p->K, p->lnN_lo, p->lnN_hi};
    return or_tab_lnp(&T, N);
}
double or_dlnp(const or_problem *p, int s, double Na, double dN)
{
    or_tab T = {p->tabL + (long)s * p->K, p->tabD1 + (long)s * p->K, p->tabD2 + (long)s * p->K,
                p->K, p->lnN_lo, p->lnN_hi};
    return or_tab_dlnp(&T, Na, dN);
}

/* Fill the rate parameters of every source for the cell at (X,Y,Z), given the
 * per-source entry columns Nin[s*ncell + gi]. */
static void cell_rates(const or_problem *p, int X, int Y, int Z, long gi, long ncell,
                       const double *Nin, or_srcrate *r)
{
    double n = p->nH[gi];
    for (int s = 0; s < p->nsrc; s++) {
        double ds, Vsh;
        src_shell(p, s, X, Y, Z, &ds, &Vsh);
        double N = Nin[(long)s * ncell + gi];
        r[s].Nin = N;
        if (p->kind[s] == 0) {
            r[s].kind = 0;
            r[s].A = p->Q[s] * exp(-p->sigma0 * N) / (n * Vsh);
            r[s].b = p->sigma0 * n * ds;
        } else {
            r[s].kind = 1;
            r[s].A = p->Q[s] / (n * Vsh);
            r[s].b = n * ds;
            r[s].tab.L = p->tabL + (long)s * p->K;
            r[s].tab.D1 = p->tabD1 + (long)s * p->K;
            r[s].tab.D2 = p->tabD2 + (long)s * p->K;
            r[s].tab.K = p->K; r[s].tab.lnN_lo = p->lnN_lo; r[s].tab.lnN_hi = p->lnN_hi;
        }
    }
}

/* Photoionisation rate per H atom (s^-1) and dx/dt of every cell for the
 * neutral fractions x and entry columns Nin (nsrc x ncell). */
void or_rates(const or_problem *p, const double *x, const double *Nin, double *F, double *xdot)
{
    long ncell = (long)p->nx * p->ny * p->nz;
    or_srcrate *r = (or_srcrate *)malloc(sizeof(or_srcrate) * (p->nsrc > 0 ? p->nsrc : 1));
    for (int Z = 0; Z < p->nz; Z++)
        for (int Y = 0; Y < p->ny; Y++)
            for (int X = 0; X < p->nx; X++) {
                long gi = X + (long)p->nx * (Y + (long)p->ny * Z);
                cell_rates(p, X, Y, Z, gi, ncell, Nin, r);
                or_cell C = {p->nsrc, r, p->alpha * p->nH[gi], 0.0};
                double Fv = cell_F(&C, x[gi]);
                if (F) F[gi] = Fv;
                if (xdot) xdot[gi] = -Fv + C.c * (1 - x[gi]) * (1 - x[gi]);
            }
    free(r);
}

/* Eq. 4 without the energy criterion: minimum over the cells with flat
 * index in [lo, hi) (all cells for the scheme, Sect. 2.2 step 2) of K1 t_rec,
 * K3 max(0.05, x)/|dx/dt|, K4/|dx/dt|. */
static double crit_dt_range(const or_problem *p, const or_scheme *sc, const double *x, const double *xdot,
                            long lo, long hi)
{
    double dt = INFINITY;
    for (long gi = lo; gi < hi; gi++) {
        if (sc->K1 > 0) {
            double v = sc->K1 / (p->alpha * p->nH[gi]);
            if (v < dt) dt = v;
        }
        if (xdot) {
            double a = fabs(xdot[gi]);
            if (a > 0) {
                if (sc->K3 > 0) {
                    double v = sc->K3 * (x[gi] > 0.05 ? x[gi] : 0.05) / a;
                    if (v < dt) dt = v;
                }
                if (sc->K4 > 0) {
                    double v = sc->K4 / a;
                    if (v < dt) dt = v;
                }
            }
        }
    }
    return dt;
}

static double crit_dt(const or_problem *p, const or_scheme *sc, const double *x, const double *xdot)
{
    return crit_dt_range(p, sc, x, xdot, 0, (long)p->nx * p->ny * p->nz);
}

/* The Eq. 4 minimum over the cells [lo, hi) for the state x and given entry
 * columns Nin (nsrc x ncell): one process's share of the cells when the
 * cells are split over processes (Sect. 5).  +inf when nothing limits it. */
double or_crit_dt_range(const or_problem *p, const or_scheme *sc, const double *x, const double *Nin, long lo, long hi)
{
    long ncell = (long)p->nx * p->ny * p->nz;
    double *xdot = (double *)malloc(sizeof(double) * ncell);
    or_rates(p, x, Nin, NULL, xdot);
    double dt = crit_dt_range(p, sc, x, xdot, lo < 0 ? 0 : lo, hi > ncell ? ncell : hi);
    free(xdot);
    return dt;
}

/* Integrate every cell from x0 over h with the entry columns Nin.  xout may
 * alias nothing; budget (if not NULL) accumulates
 *   [1] photons absorbed  sum n V IF,  [2] new ions sum n V (x0 - x),
 *   [3] recombinations sum n V IR. */
static void integrate_all(const or_problem *p, const double *x0, const double *Nin, double h,
                          double *xout, double *budget)
{
    long ncell = (long)p->nx * p->ny * p->nz;
    double V = p->dx * p->dx * p->dx;
    or_srcrate *r = (or_srcrate *)malloc(sizeof(or_srcrate) * (p->nsrc > 0 ? p->nsrc : 1));
    for (int Z = 0; Z < p->nz; Z++)
        for (int Y = 0; Y < p->ny; Y++)
            for (int X = 0; X < p->nx; X++) {
                long gi = X + (long)p->nx * (Y + (long)p->ny * Z);
                cell_rates(p, X, Y, Z, gi, ncell, Nin, r);
                or_cell C = {p->nsrc, r, p->alpha * p->nH[gi], 0.0};
                or_intres R = or_integrate_cell(&C, x0[gi], h);
                xout[gi] = R.x;
                if (budget) {
                    double nV = p->nH[gi] * V;
                    budget[1] += nV * R.IF;
                    budget[2] += nV * (x0[gi] - R.x);
                    budget[3] += nV * R.IR;
                }
            }
    free(r);
}

/*
 * Selected cells of integrate_all (Sect. 2.2: Eq. 2 over h from x0 with the
 * entry columns Nin[s*ncell + gi] frozen), for checks on grids too large to
 * integrate whole: cell idx[q] starts from x0[q]; xout[q] = x(h).
 */
void or_integrate_cells(const or_problem *p, long nq, const long *idx, const double *x0, const double *Nin,
                        double h, double *xout)
{
    long ncell = (long)p->nx * p->ny * p->nz;
    or_srcrate *r = (or_srcrate *)malloc(sizeof(or_srcrate) * (p->nsrc > 0 ? p->nsrc : 1));
    for (long q = 0; q < nq; q++) {
        long gi = idx[q];
        int X = (int)(gi % p->nx), Y = (int)((gi / p->nx) % p->ny), Z = (int)(gi / ((long)p->nx * p->ny));
        cell_rates(p, X, Y, Z, gi, ncell, Nin, r);
        or_cell C = {p->nsrc, r, p->alpha * p->nH[gi], 0.0};
        xout[q] = or_integrate_cell(&C, x0[q], h).x;
    }
    free(r);
}

/*
 * A1 (Sect. 2.1, Eq. 3), one cell: integrate (x, attenuation) over dt from
 * x0[gi] with the entry column nin frozen, store x(dt), and return the
 * effective optical depth -ln<f> at nu0 that builds the column handed
 * downstream, N_out = N_in - ln<f>/sigma0.  ds and Vsh as in src_shell.
 */
static double a1_cell(const or_problem *p, long gi, double nin, double ds, double Vsh,
                      const double *x0, double dt, double *xout, double *budget)
{
    double n = p->nH[gi];
    or_srcrate r;
    r.Nin = nin;
    if (p->kind[0] == 0) {
        r.kind = 0;
        r.A = p->Q[0] * exp(-p->sigma0 * nin) / (n * Vsh);
        r.b = p->sigma0 * n * ds;
    } else {
        r.kind = 1;
        r.A = p->Q[0] / (n * Vsh);
        r.b = n * ds;
        r.tab.L = p->tabL; r.tab.D1 = p->tabD1; r.tab.D2 = p->tabD2;
        r.tab.K = p->K; r.tab.lnN_lo = p->lnN_lo; r.tab.lnN_hi = p->lnN_hi;
    }
    or_cell C = {1, &r, p->alpha * n, p->sigma0 * n * ds};
    or_intres R = or_integrate_cell(&C, x0[gi], dt);
    xout[gi] = R.x;
    if (budget) {
        double nV = n * p->dx * p->dx * p->dx;
        budget[1] += nV * R.IF;
        budget[2] += nV * (x0[gi] - R.x);
        budget[3] += nV * R.IR;
    }
    return -R.lnfav;
}

/*
 * A1 (Sect. 2.1): one sweep per octant in which every cell, in causal order,
 * takes its entry column from the time-averaged columns of its upwind
 * neighbours, integrates (x, attenuation) over dt, and hands downstream the
 * column N_out = N_in - ln<f>/sigma0 built from its time-averaged
 * attenuation <f> at nu0 (Eq. 3).  Single source.  For a plane source the
 * causal order is along each row from the face the photons enter through.
 */
static void a1_sweep(const or_problem *p, const double *x0, double dt, double *xout,
                     double *Nin_out, double *budget)
{
    long ncell = (long)p->nx * p->ny * p->nz;
    int code = src_plane(p, 0);
    if (code >= 0) {
        int n3[3] = {p->nx, p->ny, p->nz};
        int axis = code / 2;
        for (int w = 0; w < n3[(axis + 2) % 3]; w++)
            for (int u = 0; u < n3[(axis + 1) % 3]; u++) {
                double N = 0.0;
                for (int m = 0; m < n3[axis]; m++) {
                    long gi = plane_cell(p, code, m, u, w);
                    if (Nin_out) Nin_out[gi] = N;
                    N += a1_cell(p, gi, N, p->dx, p->dx, x0, dt, xout, budget) / p->sigma0;
                }
            }
        return;
    }
    double *Nout = (double *)malloc(sizeof(double) * ncell);
    double *dtau = (double *)malloc(sizeof(double) * ncell);
    const int *v = p->vtx;
    int n3[3] = {p->nx, p->ny, p->nz};
    for (int oct = 0; oct < 8; oct++) {
        int sg[3] = {(oct & 1) ? -1 : 1, (oct & 2) ? -1 : 1, (oct & 4) ? -1 : 1};
        int ext[3];
        for (int q = 0; q < 3; q++) ext[q] = sg[q] > 0 ? n3[q] - v[q] : v[q];
        if (ext[0] <= 0 || ext[1] <= 0 || ext[2] <= 0) continue;
        int mmax = ext[0] + ext[1] + ext[2] - 3;
        for (int m = 0; m <= mmax; m++) {
            for (int i = 0; i < ext[0] && i <= m; i++) {
                for (int j = 0; j < ext[1] && i + j <= m; j++) {
                    int k = m - i - j;
                    if (k >= ext[2]) continue;
                    int G[3] = {sg[0] > 0 ? v[0] + i : v[0] - 1 - i,
                                sg[1] > 0 ? v[1] + j : v[1] - 1 - j,
                                sg[2] > 0 ? v[2] + k : v[2] - 1 - k};
                    long gi = G[0] + (long)p->nx * (G[1] + (long)p->ny * G[2]);
                    double nin = (m == 0) ? 0.0 : sc_interp(p, v, sg, ext, i, j, k, Nout, dtau);
                    double ds, Vsh;
                    src_shell(p, 0, G[0], G[1], G[2], &ds, &Vsh);
                    double dtau_eff = a1_cell(p, gi, nin, ds, Vsh, x0, dt, xout, budget);
                    if (Nin_out) Nin_out[gi] = nin;
                    Nout[gi] = nin + dtau_eff / p->sigma0;
                    dtau[gi] = dtau_eff;
                }
            }
        }
    }
    free(Nout);
    free(dtau);
}

/*
 * One substep of the chosen scheme, advancing x in place from t to t + dt
 * (dt from Eq. 4 or fixed, capped at t_end - t).  Returns dt.
 *   budget (4 doubles, overwritten): emitted photons (sum Q dt; a plane
 *   source's flux times its entry face), absorbed, new ions,
 *   recombinations (the last three from the full-step integration);
 *   Nin1 (optional, nsrc x ncell): the entry columns of the first trace.
 * A3 (Sect. 2.2, Fig. 1): trace x^n; dt; x_half = X(x^n, N^1, dt/2); trace
 *   x_half; x^{n+1} = X(x^n, N^{1/2}, dt).
 * A2: trace x^n; dt; x^{n+1} = X(x^n, N^1, dt).
 * A1: dt (K1 t_rec; a trace of x^n first if K3 or K4 is used); implicit sweep.
 */
double or_substep(const or_problem *p, const or_scheme *sc, double *x, double *t, double t_end,
                  double *budget, double *Nin1)
{
    long ncell = (long)p->nx * p->ny * p->nz;
    int S = p->nsrc;
    double *N1 = Nin1 ? Nin1 : (double *)malloc(sizeof(double) * ncell * (S > 0 ? S : 1));
    double *xdot = (double *)malloc(sizeof(double) * ncell);
    double bud[4] = {0, 0, 0, 0};
    int need_trace = (sc->scheme != 1) || (sc->dt_fixed <= 0 && (sc->K3 > 0 || sc->K4 > 0));
    if (need_trace)
        for (int s = 0; s < S; s++) or_trace(p, s, x, N1 + (long)s * ncell, NULL);
    double dt;
    if (sc->dt_fixed > 0) dt = sc->dt_fixed;
    else {
        if (need_trace) or_rates(p, x, N1, NULL, xdot);
        dt = crit_dt(p, sc, x, need_trace ? xdot : NULL);
    }
    if (dt > t_end - *t) dt = t_end - *t;
    if (!(dt > 0)) dt = 0;
    double *xn = (double *)malloc(sizeof(double) * ncell);
    if (sc->scheme == 3) {
        double *xh = (double *)malloc(sizeof(double) * ncell);
        double *N2 = (double *)malloc(sizeof(double) * ncell * (S > 0 ? S : 1));
        integrate_all(p, x, N1, 0.5 * dt, xh, NULL);
        for (int s = 0; s < S; s++) or_trace(p, s, xh, N2 + (long)s * ncell, NULL);
        integrate_all(p, x, N2, dt, xn, bud);
        free(xh);
        free(N2);
    } else if (sc->scheme == 2) {
        integrate_all(p, x, N1, dt, xn, bud);
    } else {
        a1_sweep(p, x, dt, xn, (need_trace || !Nin1) ? NULL : N1, bud);
    }
    for (int s = 0; s < S; s++) bud[0] += src_emission(p, s) * dt;
    memcpy(x, xn, sizeof(double) * ncell);
    *t += dt;
    if (budget) memcpy(budget, bud, sizeof(bud));
    free(xn);
    free(xdot);
    if (!Nin1) free(N1);
    return dt;
}

/*
 * Brute-force long characteristics: the exact column of neutral hydrogen
 * along the straight segment from source s's vertex to the centre of every
 * cell, by exact voxel traversal of the segment (accumulating n x times the
 * length inside each voxel).
 */
void or_long_char(const or_problem *p, int s, const double *x, double *Ncentre)
{
    if (src_plane(p, s) >= 0) {
        /* the ray to a cell centre runs along its row: whole cells before it,
         * half of its own */
        long ncell = (long)p->nx * p->ny * p->nz;
        or_trace(p, s, x, Ncentre, NULL);
        for (long gi = 0; gi < ncell; gi++) Ncentre[gi] += 0.5 * p->nH[gi] * x[gi] * p->dx;
        return;
    }
    const int *v = p->vtx + 3 * s;
    int n3[3] = {p->nx, p->ny, p->nz};
    for (int Z = 0; Z < p->nz; Z++)
        for (int Y = 0; Y < p->ny; Y++)
            for (int X = 0; X < p->nx; X++) {
                long gi = X + (long)p->nx * (Y + (long)p->ny * Z);
                double P0[3] = {(double)v[0], (double)v[1], (double)v[2]};
                double P1[3] = {X + 0.5, Y + 0.5, Z + 0.5};
                double d[3];
                for (int q = 0; q < 3; q++) d[q] = P1[q] - P0[q];
                /* parametric crossings t in (0,1) of integer planes along each axis */
                double ts[3 * 2048 + 2];
                int nt = 0;
                ts[nt++] = 0.0;
                for (int q = 0; q < 3; q++) {
                    if (d[q] == 0.0) continue;
                    double a = P0[q], b = P1[q];
                    int lo = (int)ceil(fmin(a, b)), hi = (int)floor(fmax(a, b));
                    for (int m = lo; m <= hi && nt < 3 * 2048; m++) {
                        double tt = (m - a) / d[q];
                        if (tt > 0.0 && tt < 1.0) ts[nt++] = tt;
                    }
                }
                ts[nt++] = 1.0;
                /* insertion sort (short lists) */
                for (int a = 1; a < nt; a++) {
                    double key = ts[a];
                    int b = a - 1;
                    while (b >= 0 && ts[b] > key) { ts[b + 1] = ts[b]; b--; }
                    ts[b + 1] = key;
                }
                double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * p->dx;
                double col = 0.0;
                for (int a = 0; a + 1 < nt; a++) {
                    double dt = ts[a + 1] - ts[a];
                    if (dt <= 0) continue;
                    double tm = 0.5 * (ts[a] + ts[a + 1]);
                    int C[3];
                    int ok = 1;
                    for (int q = 0; q < 3; q++) {
                        C[q] = (int)floor(P0[q] + tm * d[q]);
                        if (C[q] < 0 || C[q] >= n3[q]) ok = 0;
                    }
                    if (!ok) continue;
                    long ci = C[0] + (long)p->nx * (C[1] + (long)p->ny * C[2]);
                    col += p->nH[ci] * x[ci] * dt * len;
                }
                Ncentre[gi] = col;
            }
}

/* Source position (in cell units) moved to the nearest cell vertex
 * (Sect. 5: the source is moved to the nearest vertex for raytracing),
 * halves rounded up, clamped to the grid's vertex range [0, n]. */
int or_snap(double pos, int n)
{
    double v = floor(pos + 0.5);
    if (v < 0) v = 0;
    if (v > n) v = n;
    return (int)v;
}

/* The timestep interface (Sect. 2.1): trace x for every source and return the
 * Eq. 4 minimum over all cells (+inf when no criterion limits it). */
double or_compute_dt(const or_problem *p, const or_scheme *sc, const double *x)
{
    long ncell = (long)p->nx * p->ny * p->nz;
    int S = p->nsrc;
    double *N1 = (double *)malloc(sizeof(double) * ncell * (S > 0 ? S : 1));
    double *xdot = (double *)malloc(sizeof(double) * ncell);
    for (int s = 0; s < S; s++) or_trace(p, s, x, N1 + (long)s * ncell, NULL);
    or_rates(p, x, N1, NULL, xdot);
    double dt = crit_dt(p, sc, x, xdot);
    free(N1);
    free(xdot);
    return dt;
}
