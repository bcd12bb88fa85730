// Per-cell passes of a substep (Mackey 2012, Sect. 2.2): the timestep
// criterion of Eq. 4 (minimum over all cells), the half-step and full-step
// integrations of Eq. 2 with frozen entry columns, and the photon budget.
// Elementwise over every cell of every grid of the call; one flat index space,
// grids located by binary search over their cell offsets.
//
// The integrations run in two passes.  The first pass settles every cell that
// a closed form covers (photon-free, at its root, or slow enough for the
// linearised step: almost all of them) and appends the others to a queue.
// The second pass gives each queued cell a whole warp: the quadrature nodes
// of every panel are evaluated one per lane, so the few slow cells near the
// ionisation front neither hold up warps of fast cells nor run their node
// evaluations one after another.
#include <algorithm>

#include "common.cuh"
#include "integrator.cuh"
#include "kernels.h"

namespace oots {

// general-pass queue record of a single-source cell: x0, n, A, b, N_in, p, F(x0), F'(x0), f(x0)
constexpr int QREC = 9;

__device__ __forceinline__ int find_grid(const long long *off, int ngrid, long long idx)
{
    int lo = 0, hi = ngrid - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Whether the pass has work on grids lo..hi: the Eq. 4 pass on a grid that
// has not reached its end time, an integration on a grid with a step in
// flight.  Blocks of grids past their end return at once, so substeps
// enqueued beyond the end cost little.
template <typename Real, int OP>
__device__ __forceinline__ bool cells_live(const GridDev<Real> *grids, int lo, int hi)
{
    for (int q = lo; q <= hi; q++) {
        const DevState *sq = grids[q].st;
        if (OP == OP_RATEDT ? !sq->done : sq->dt > 0.0) return true;
    }
    return false;
}

// Rate parameters of every source for the cell at global index g = (X,Y,Z).
// with_p = false leaves r[s].p of tabulated sources to the caller.
template <typename Real, int NSMAX>
__device__ __forceinline__ int cell_rates(const GridDev<Real> &G, const Real *Ncol, const DevTable<Real> *tabs,
                                          int X, int Y, int Z, long long g, Real n, SrcRate<Real> *r,
                                          bool with_p = true)
{
    for (int s = 0; s < NSMAX && s < G.nsrc; s++) {
        const int i = X >= G.vtx[s][0] ? X - G.vtx[s][0] : G.vtx[s][0] - 1 - X;
        const int j = Y >= G.vtx[s][1] ? Y - G.vtx[s][1] : G.vtx[s][1] - 1 - Y;
        const int k = Z >= G.vtx[s][2] ? Z - G.vtx[s][2] : G.vtx[s][2] - 1 - Z;
        src_rate<Real>(r[s], G.qfac[s], G.tab[s], G.sigma0, G.dx, n, G.pcode[s] != 0, i, j, k,
                       Ncol[(long long)s * G.ncell + g], tabs, with_p);
    }
    return G.nsrc;
}

// Mixed path: warp sums of two FP32 values, scaled to FP64 once per warp,
// then the block sum in FP64; thread 0 gets both (one pair of barriers).
__device__ __forceinline__ void block_sum2_f(float a, float b, double scale, double &ra, double &rb, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sh[2 * wid] = double(a) * scale; sh[2 * wid + 1] = double(b) * scale; }
    __syncthreads();
    if (threadIdx.x == 0) {
        ra = 0.0; rb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { ra += sh[2 * w]; rb += sh[2 * w + 1]; }
    }
}

// Block sums of two values in one pass (one pair of barriers); thread 0 gets both.
__device__ __forceinline__ void block_sum2(double &a, double &b, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) { sh[2 * wid] = a; sh[2 * wid + 1] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0; b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { a += sh[2 * w]; b += sh[2 * w + 1]; }
    }
}

template <typename Real, int OP, int NSMAX, int BS>
__global__ void __launch_bounds__(BS, 1024 / BS) cell_kernel(const GridDev<Real> *grids, int ngrid, const long long *offsets,
                                                   long long total, const DevTable<Real> *tabs, unsigned *queue,
                                                   unsigned *qcount, Real *qrec, Real *rcache, int use_cache)
{
    __shared__ double sh[32];
    __shared__ int s_grid_lo, s_grid_hi;
    const long long base = (long long)blockIdx.x * blockDim.x;
    // every thread of a block works on one grid at a time; a block straddling
    // two grids loops over both (the reductions are per grid)
    if (threadIdx.x == 0) {
        long long last = base + blockDim.x - 1;
        if (last >= total) last = total - 1;
        s_grid_lo = find_grid(offsets, ngrid, base < total ? base : total - 1);
        s_grid_hi = find_grid(offsets, ngrid, last);
        if (!cells_live<Real, OP>(grids, s_grid_lo, s_grid_hi)) s_grid_hi = s_grid_lo - 1;
    }
    __syncthreads();
    // mixed path: the step and the Eq. 4 factors in FP32, converted once per
    // block (this GPU runs FP64 at a small fraction of its FP32 rate, so the
    // per-cell criterion and budget stay off the FP64 pipe)
    constexpr bool F32 = sizeof(Real) == 4;
    __shared__ float s_f[4];
    for (int gi = s_grid_lo; gi <= s_grid_hi; gi++) {
        const GridDev<Real> &G = grids[gi];
        DevState *st = G.st;
        const long long idx = base + threadIdx.x;
        const bool mine = idx < total && idx >= offsets[gi] && (gi + 1 >= ngrid || idx < offsets[gi + 1]) &&
                          idx - offsets[gi] >= G.cell_lo && idx - offsets[gi] < G.cell_hi;
        if (F32) {
            if (threadIdx.x == 0) {
                const double d = st->dt;
                s_f[0] = float(OP == OP_HALF ? 0.5 * d : d);
                s_f[1] = float(st->K1);
                s_f[2] = float(st->K3);
                s_f[3] = float(st->K4);
            }
            __syncthreads();
        }
        const double dtd = F32 ? 0.0 : st->dt;
        const bool stepping = F32 ? s_f[0] > 0.0f : dtd > 0.0;
        const bool active = mine && (OP == OP_RATEDT || stepping) && !(OP == OP_RATEDT && st->done);
        double dtmin = __longlong_as_double(0x7ff0000000000000ll);
        float dtmin_f = __int_as_float(0x7f800000);
        double ions = 0.0, rec = 0.0;
        float ions_f = 0.0f, rec_f = 0.0f;
        bool defer = false;
        Real rv[QREC];
        if (active) {
            const long long g = idx - offsets[gi];
            const int X = (int)(g % G.nx);
            const int Y = (int)((g / G.nx) % G.ny);
            const int Z = (int)(g / ((long long)G.nx * G.ny));
            const Real n = G.n ? G.n[g] : G.n_uniform;
            const Real x0 = G.x[g];
            SrcRate<Real> r[NSMAX];
            const Real *Ncol = (OP == OP_FULL2) ? G.N2 : G.N1;
            CellODE<Real> C;
            // single source, same state and columns as this substep's dt pass:
            // its transmitted fraction and F, F' at x0 come from the rate cache
            const bool cached = NSMAX == 1 && (OP == OP_HALF || OP == OP_FULL1) && use_cache;
            C.ns = cell_rates<Real, NSMAX>(G, Ncol, tabs, X, Y, Z, g, n, r, !cached);
            if (cached && C.ns > 0) r[0].p = rcache[idx];
            C.c = G.alpha * n;
            C.b0 = Real(0);
            C.r = r;
            C.tabs = tabs;
            if (OP == OP_RATEDT) {
                // Eq. 4 with T fixed: K1 t_rec, K3 max(0.05, x)/|dx/dt|, K4/|dx/dt|
                Real F, dF;
                ode_F<Real, NSMAX>(C, x0, &F, &dF);
                if (NSMAX == 1 && rcache && C.ns > 0) {
                    rcache[idx] = r[0].p;
                    rcache[total + idx] = F;
                    rcache[2 * total + idx] = dF;
                }
                if (F32) {
                    const float xd = fabsf(float(-F + C.c * (Real(1) - x0) * (Real(1) - x0)));
                    if (s_f[1] > 0.0f) dtmin_f = fminf(dtmin_f, s_f[1] / (float(G.alpha) * float(n)));
                    if (xd > 0.0f) {
                        if (s_f[2] > 0.0f) dtmin_f = fminf(dtmin_f, s_f[2] * fmaxf(0.05f, float(x0)) / xd);
                        if (s_f[3] > 0.0f) dtmin_f = fminf(dtmin_f, s_f[3] / xd);
                    }
                } else {
                    const double xd = fabs((double)(-F + C.c * (Real(1) - x0) * (Real(1) - x0)));
                    if (st->K1 > 0) dtmin = fmin(dtmin, st->K1 / (double(G.alpha) * double(n)));
                    if (xd > 0) {
                        if (st->K3 > 0) dtmin = fmin(dtmin, st->K3 * fmax(0.05, (double)x0) / xd);
                        if (st->K4 > 0) dtmin = fmin(dtmin, st->K4 / xd);
                    }
                }
            } else {
                // closed forms here; the rest goes to the warp-per-cell pass
                IntResult<Real> R;
                Real F0 = Real(0), dF0 = Real(0), f0;
                const Real h = F32 ? Real(s_f[0]) : Real(OP == OP_HALF ? 0.5 * dtd : dtd);
                if (cached && C.ns > 0) { F0 = rcache[total + idx]; dF0 = rcache[2 * total + idx]; }
                if (integrate_prelude<Real, NSMAX>(C, x0, h, G.sigma0, R, F0, dF0, f0, cached && C.ns > 0)) {
                    if (OP == OP_HALF) {
                        const_cast<Real *>(G.xh)[g] = R.x;
                    } else {
                        G.xout[g] = R.x;
                        if (F32) {
                            // per H atom times n; the cell volume is applied per warp
                            ions_f = float(n) * (float(x0) - float(R.x));
                            rec_f = float(n) * float(R.IR);
                        } else {
                            const double nV = double(n) * st->cell_volume;
                            ions = nV * (double(x0) - double(R.x));
                            rec = nV * double(R.IR);
                        }
                    }
                } else {
                    defer = true;
                    if (NSMAX == 1) {
                        // what the general pass would otherwise recompute
                        rv[0] = x0; rv[1] = n; rv[2] = r[0].A; rv[3] = r[0].b; rv[4] = r[0].Nin; rv[5] = r[0].p;
                        rv[6] = F0; rv[7] = dF0; rv[8] = f0;
                    }
                }
            }
        }
        if (OP != OP_RATEDT) {
            // warp-aggregated append to the queue of the general pass
            const unsigned m = __ballot_sync(0xffffffffu, defer);
            if (m) {
                const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                unsigned base = 0;
                if (lane == leader) base = atomicAdd(qcount + (OP == OP_HALF ? 0 : 1), (unsigned)__popc(m));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (defer) {
                    const unsigned slot = base + __popc(m & ((1u << lane) - 1u));
                    queue[slot] = (unsigned)idx;
                    if (NSMAX == 1)
#pragma unroll
                        for (int v = 0; v < QREC; v++) qrec[(size_t)slot * QREC + v] = rv[v];
                }
            }
        }
        if (OP == OP_RATEDT) {
            if (F32) {
                for (int o = 16; o > 0; o >>= 1) dtmin_f = fminf(dtmin_f, __shfl_down_sync(0xffffffffu, dtmin_f, o));
                if ((threadIdx.x & 31) == 0) dtmin = double(dtmin_f);   // lane 0 carries the warp minimum
            } else {
                for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_down_sync(0xffffffffu, dtmin, o));
            }
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            __syncthreads();
            if (lane == 0) sh[wid] = dtmin;
            __syncthreads();
            if (threadIdx.x == 0) {
                double m = sh[0];
                for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmin(m, sh[w]);
                // (the read skips the atomic of a block that cannot lower the minimum)
                const unsigned long long mb = (unsigned long long)__double_as_longlong(m);
                if (m < 1e300 && mb < *(volatile unsigned long long *)&st->dt_bits) atomicMin(&st->dt_bits, mb);
            }
        } else if (OP == OP_FULL1 || OP == OP_FULL2) {
            double si = ions, sr = rec;
            if (F32) block_sum2_f(ions_f, rec_f, st->cell_volume, si, sr, sh);
            else block_sum2(si, sr, sh);
            if (threadIdx.x == 0 && (si != 0.0 || sr != 0.0)) {
                atomicAdd(&st->bud_step[1], si + sr);   // absorbed = new ions + recombinations
                atomicAdd(&st->bud_step[2], si);
                atomicAdd(&st->bud_step[3], sr);
            }
        }
        __syncthreads();
    }
}

// General pass: one lane group per queued cell (a half warp in FP32, a warp
// in FP64; HALF: queue 0, FULL: queue 1).  Groups take the next queued cell
// from a head counter (qcount[2 + queue]), so the pass ends when the cells
// run out rather than when the group that drew the slowest share finishes.
// Every lane forms the same rates and runs the same root search; the
// quadrature nodes are spread over the lanes (WarpEval).  Budget sums of FULL
// are gathered per block in shared memory for up to eight grids and flushed
// with one atomic per grid and block.
template <typename Real, int OP, int NSMAX>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 4 : 2)
cell_general_kernel(const GridDev<Real> *grids, int ngrid, const long long *offsets, const DevTable<Real> *tabs,
                    const unsigned *queue, unsigned *qcount, const Real *qrec)
{
    __shared__ double s_ions[8], s_rec[8];
    __shared__ int s_gid[8];
    constexpr int W = GroupWidth<Real>::value;
    const int lane32 = threadIdx.x & 31;
    const int gbase = lane32 & ~(W - 1), lane = lane32 - gbase;
    const unsigned gmask = W == 32 ? 0xffffffffu : (0xffffu << gbase);
    if (OP != OP_HALF) {
        if (threadIdx.x < 8) { s_ions[threadIdx.x] = 0.0; s_rec[threadIdx.x] = 0.0; s_gid[threadIdx.x] = -1; }
        __syncthreads();
    }
    const int qi = OP == OP_HALF ? 0 : 1;
    const unsigned nq = qcount[qi];
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(&qcount[2 + qi], 1u);
        q = __shfl_sync(gmask, q, gbase);
        if (q >= nq) break;
        const long long idx = queue[q];
        const int gi = find_grid(offsets, ngrid, idx);
        const GridDev<Real> &G = grids[gi];
        DevState *st = G.st;
        const double dtd = st->dt;
        const long long g = idx - offsets[gi];
        SrcRate<Real> r[NSMAX];
        CellODE<Real> C;
        Real n, x0, F0, dF0, f0;
        IntResult<Real> R;
        const Real h = Real(OP == OP_HALF ? 0.5 * dtd : dtd);
        bool done = false;
        if (NSMAX == 1) {
            // one source: the closed-form pass left its rates and f(x0)
            const Real *rv = qrec + (size_t)q * QREC;
            x0 = rv[0]; n = rv[1];
            r[0].A = rv[2]; r[0].b = rv[3]; r[0].Nin = rv[4]; r[0].p = rv[5]; r[0].tab = G.tab[0];
            F0 = rv[6]; dF0 = rv[7]; f0 = rv[8];
            C.ns = 1;
            R.x = x0; R.IR = Real(0); R.lnfav = Real(0);
        } else {
            const int X = (int)(g % G.nx);
            const int Y = (int)((g / G.nx) % G.ny);
            const int Z = (int)(g / ((long long)G.nx * G.ny));
            n = G.n ? G.n[g] : G.n_uniform;
            x0 = G.x[g];
            const Real *Ncol = (OP == OP_FULL2) ? G.N2 : G.N1;
            C.ns = cell_rates<Real, NSMAX>(G, Ncol, tabs, X, Y, Z, g, n, r);
        }
        C.c = G.alpha * n;
        C.b0 = Real(0);
        C.r = r;
        C.tabs = tabs;
        if (NSMAX != 1) done = integrate_prelude<Real, NSMAX>(C, x0, h, G.sigma0, R, F0, dF0, f0);
        if (!done)
            R = integrate_general<Real, NSMAX>(C, x0, h, G.sigma0, R, F0, dF0, f0, GroupEval<W>{lane, gbase, gmask});
        if (lane == 0) {
            if (OP == OP_HALF) {
                const_cast<Real *>(G.xh)[g] = R.x;
            } else {
                G.xout[g] = R.x;
                const double nV = double(n) * st->cell_volume;
                const double ions = nV * (double(x0) - double(R.x)), rec = nV * double(R.IR);
                const int slot = gi & 7;
                const int owner = atomicCAS(&s_gid[slot], -1, gi);
                if (owner == -1 || owner == gi) {
                    atomicAdd(&s_ions[slot], ions);
                    atomicAdd(&s_rec[slot], rec);
                } else {
                    atomicAdd(&st->bud_step[1], ions + rec);
                    atomicAdd(&st->bud_step[2], ions);
                    atomicAdd(&st->bud_step[3], rec);
                }
            }
        }
    }
    if (OP != OP_HALF) {
        __syncthreads();
        if (threadIdx.x < 8 && s_gid[threadIdx.x] >= 0) {
            DevState *st = grids[s_gid[threadIdx.x]].st;
            atomicAdd(&st->bud_step[1], s_ions[threadIdx.x] + s_rec[threadIdx.x]);
            atomicAdd(&st->bud_step[2], s_ions[threadIdx.x]);
            atomicAdd(&st->bud_step[3], s_rec[threadIdx.x]);
        }
    }
}

// ---------------------------------------------------------------------------
// Many sources per grid: per-cell source selection
// ---------------------------------------------------------------------------
// A source can raise a cell's photoionisation rate per unit neutral fraction
// by at most amp = A b (monochromatic) or A p sigma0 b (tabulated: no
// cross-section exceeds sigma0).  Both equal qfac sigma0 dx p / r2 (r2 = 1 for
// a plane source), p the fraction of the source's photons that reach the
// cell.  A source with amp h at most a thousandth of the rounding cannot move
// x over a step h, so it is left out of the cell's rate (the rule by which the
// single-source closed forms call a cell photon-free).  The bound is formed in
// float, from the table node at or below the column (P falls as N grows); the
// rates of the sources kept are then formed exactly, in a few registers.
constexpr int NACT = 4;        // sources the closed-form passes hold in registers

// The entry column beyond which source s cannot reach the threshold e^lnthr at
// any cell: r2 >= 3/4, so amp <= e^lnthr whenever ln P/Q <= lnthr - ln(qfac
// sigma0 dx) + ln(3/4).  Monochromatic: ln P/Q = -sigma0 N.  Tabulated: the
// bound (sel_lnamp) reads the node one interval below N, so N at or above the
// node after the first node below the target qualifies.  +inf: never.
template <typename Real>
__device__ Real negligible_column(const GridDev<Real> &G, const DevTable<Real> *tabs, int s, float lnthr)
{
    const float target = lnthr - G.lnamp0[s] + -0.2876821f;          // ln(3/4)
    if (!(target > -1e30f)) return RealLimits<Real>::inf();        // lnthr = -inf: keep everything
    if (target >= 0.0f) return Real(0);                            // never above the threshold
    if (G.tab[s] < 0) return Real(-target) / G.sigma0;
    const DevTable<Real> &T = tabs[G.tab[s]];
    // first node with L <= target (L falls with the node index)
    int lo = 0, hi = T.K;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (float(T.L[mid]) <= target) hi = mid; else lo = mid + 1;
    }
    if (lo + 1 >= T.K) return T.Nhi;                                // beyond the table P = 0
    return T.Nnode[lo + 1];
}

// ln of the bound amp of one source at cell (X, Y, Z) with entry column N,
// from the source's record, and the cell's octant-local indices (i, j, k).
// r2 = |c|^2 in units of dx^2 (1 for a plane source, whose rate shares
// photons per unit area); ln P/Q rounded up: -sigma0 N (monochromatic) or the
// table node one interval below N's (tabulated; 0 below the table, -inf
// above it).
template <typename Real>
__device__ __forceinline__ float sel_lnamp(const SrcSel<Real> &S, int X, int Y, int Z, Real N, int &i, int &j, int &k)
{
    i = X >= S.v0 ? X - S.v0 : S.v0 - 1 - X;
    j = Y >= S.v1 ? Y - S.v1 : S.v1 - 1 - Y;
    k = Z >= S.v2 ? Z - S.v2 : S.v2 - 1 - Z;
    float r2 = 1.0f;
    if (!S.plane) {
        const float c0 = i + 0.5f, c1 = j + 0.5f, c2 = k + 0.5f;
        r2 = c0 * c0 + c1 * c1 + c2 * c2;
    }
    float lnp;
    if (S.K < 0) {
        lnp = S.msig * (float)N;
    } else if (!(N > S.N0)) {
        lnp = 0.0f;
    } else if (N > S.Nhi) {
        lnp = -__int_as_float(0x7f800000);
    } else {
        int kk = (int)floorf((__logf((float)N) - S.lnN_lo) * S.inv_dl) - 1;
        kk = kk < 0 ? 0 : (kk > S.K - 1 ? S.K - 1 : kk);
        lnp = (float)S.L[kk];
    }
    return S.lnamp0 + lnp - __logf(r2);
}

// The entry columns of sources s0 .. s0+7 at cell g, loaded together (eight
// loads in flight instead of one latency per source).
template <typename Real>
__device__ __forceinline__ void load_columns8(const GridDev<Real> &G, const Real *Ncol, int s0, long long g, Real *Nb)
{
#pragma unroll
    for (int q = 0; q < 8; q++) Nb[q] = s0 + q < G.nsrc ? Ncol[(long long)(s0 + q) * G.ncell + g] : Real(0);
}

// Rate parameters of the sources whose bound exceeds e^lnthr, into
// r[0 .. NK-1] (indices fixed at compile time, so r stays in registers).
// Returns how many there are; NK + 1 when there are more than NK.  sel: the
// pass's source records; a source whose entry column is at or beyond its
// record's negligible column is left out without forming its bound.
template <typename Real, int NK>
__device__ __forceinline__ int gather_rates_sel(const GridDev<Real> &G, const SrcSel<Real> *sel, const Real *Ncol,
                                                const DevTable<Real> *tabs, int X, int Y, int Z, long long g, Real n,
                                                float lnthr, SrcRate<Real> *r)
{
    int cnt = 0;
    for (int s0 = 0; s0 < G.nsrc; s0 += 8) {
        Real Nb[8];
        load_columns8(G, Ncol, s0, g, Nb);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int s = s0 + q;
            if (s >= G.nsrc) break;
            const Real N = Nb[q];
            const SrcSel<Real> &S = sel[s];
            if (N >= S.nst) continue;
            int i, j, k;
            if (!(sel_lnamp(S, X, Y, Z, N, i, j, k) > lnthr)) continue;
            if (cnt == NK) return NK + 1;
            SrcRate<Real> t;
            src_rate<Real>(t, G.qfac[s], G.tab[s], G.sigma0, G.dx, n, G.pcode[s] != 0, i, j, k, N, tabs);
            if constexpr (NK <= 16) {
#pragma unroll
                for (int u = 0; u < NK; u++)
                    if (u == cnt) r[u] = t;
            } else {
                r[cnt] = t;                 // a local-memory array: index it directly
            }
            cnt++;
        }
    }
    return cnt;
}

// ln(1e-3 eps / h): the selection threshold for a step h (-inf: keep every source)
template <typename Real> __device__ __forceinline__ float lnthr_step(double h)
{
    if (!(h > 0.0) || !(h < 1e290)) return -__int_as_float(0x7f800000);
    return (float)(log(1e-3 * (double)RealLimits<Real>::eps()) - log(h));
}

// Closed forms from F(x0), F'(x0) alone (no per-source rates): photon-free,
// at the root within rounding, or slow enough for the linearised step.  bm
// bounds the optical-depth scale of every source per unit x.  Returns true
// when the cell is done.
template <typename Real>
__device__ __forceinline__ bool closed_form_from_F(Real c, Real x0, Real h, Real F0, Real dF0, Real bm,
                                                   IntResult<Real> &R)
{
    const Real f0 = -F0 + c * (Real(1) - x0) * (Real(1) - x0);
    if (m_abs(f0) <= Real(32) * RealLimits<Real>::eps() * (m_abs(F0) + c * (Real(1) - x0) * (Real(1) - x0))) {
        R.x = x0;
        R.IR = h * c * (Real(1) - x0) * (Real(1) - x0);
        return true;
    }
    const Real df0 = -dF0 - Real(2) * c * (Real(1) - x0);
    const Real z = h * df0;
    if (!(m_abs(z) <= IntCfg<Real>::zlin())) return false;
    const Real phi = (m_abs(z) > Real(1e-8)) ? m_expm1(z) / z : Real(1) + Real(0.5) * z;
    const Real dx = h * f0 * phi;
    const Real adx = m_abs(dx);
    if (bm * adx <= IntCfg<Real>::zlin() && c * h * adx <= IntCfg<Real>::zlin() * IntCfg<Real>::zlin() &&
        x0 + dx >= Real(0) && x0 + dx <= Real(1)) {
        R.x = x0 + dx;
        const Real xm = x0 + Real(0.5) * dx;
        R.IR = h * c * (Real(1) - xm) * (Real(1) - xm);
        return true;
    }
    return false;
}

// Per-cell passes of grids with several sources.
//
// RATEDT (Eq. 4 minimum over cells) bounds every source's rate at the cell
// against a hint H of the step (four times the last substep's) and forms the
// exact F and F' from the sources whose bound times H exceeds a thousandth
// of the rounding; a cell that no source reaches so is photon-free within H
// (F = F' = 0) and only recombines.  Left-out sources change the limiting
// |dx/dt| by far less than its rounding as long as the step comes out below
// H; a second, verifying launch (verify = 1) recomputes every cell without
// hint when it did not, and returns at once otherwise.  Per source, a column
// beyond which it cannot reach the threshold anywhere (SrcSel::nst, set by the
// finalize kernel once per substep) skips even the bound.  RATEDT caches F,
// F' and the sum of the bounds for the step that follows on the same columns
// (A3's half step, A2's full step), which settles photon-free and slow cells
// from the cache alone.  A3's full step (new columns) and the cells the cache
// does not settle select their sources for the step and run the closed forms
// on them; the rest go to the general pass.  The kernel walks BS-cell
// chunks with a stride of the grid size.
// BS: threads (and cells) per block, 128 or 256 (tuned): small blocks hold up
// fewer cells at their barriers behind a slow one.
template <typename Real, int OP, int BS>
__global__ void __launch_bounds__(BS, (sizeof(Real) == 4 ? 1024 : 512) / BS) cell_multi_kernel(const GridDev<Real> *grids, int ngrid,
                                                         const long long *offsets, long long total,
                                                         const DevTable<Real> *tabs, unsigned *queue,
                                                         unsigned *qcount, Real *rcache, int use_cache, int verify)
{
    __shared__ double sh[32];
    __shared__ int s_grid_lo, s_grid_hi, s_skip;
    __shared__ double s_h, s_hint;
    __shared__ float s_lnthr, s_f[4];
    constexpr bool F32 = sizeof(Real) == 4;
    const long long nchunk = (total + BS - 1) / BS;
    if (OP == OP_RATEDT && verify) {
        // nothing to do unless some grid's first-pass minimum exceeded its hint
        if (threadIdx.x == 0) {
            int any = 0;
            for (int q = 0; q < ngrid && !any; q++) {
                const DevState *sq = grids[q].st;
                const double d = sq->dt_last;
                const unsigned long long b = sq->dt_bits;
                if (sq->done || !(d > 0.0)) continue;            // no hint was used
                any = b == 0xffffffffffffffffull || __longlong_as_double((long long)b) > 4.0 * d;
            }
            s_skip = any;
        }
        __syncthreads();
        if (!s_skip) return;
    }
    for (long long chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x) {
    const long long base = chunk * BS;
    if (threadIdx.x == 0) {
        long long last = base + blockDim.x - 1;
        if (last >= total) last = total - 1;
        s_grid_lo = find_grid(offsets, ngrid, base);
        s_grid_hi = find_grid(offsets, ngrid, last);
        if (!cells_live<Real, OP>(grids, s_grid_lo, s_grid_hi)) s_grid_hi = s_grid_lo - 1;
    }
    __syncthreads();
    for (int gi = s_grid_lo; gi <= s_grid_hi; gi++) {
        const GridDev<Real> &G = grids[gi];
        DevState *st = G.st;
        if (threadIdx.x == 0) {
            const double d = st->dt;
            const double h = OP == OP_HALF ? 0.5 * d : d;
            s_h = h;
            s_skip = 0;
            if (OP == OP_RATEDT) {
                // the last substep's step (st->dt of this substep is not chosen yet)
                const double dl = st->dt_last;
                double hint = dl > 0.0 ? 4.0 * dl : __longlong_as_double(0x7ff0000000000000ll);
                if (verify) {
                    // a minimum at or below the hint stands: every cell the first pass
                    // skipped asks for more.  (Other blocks of this pass may have lowered
                    // it meanwhile; that only means the same.)
                    const unsigned long long b = st->dt_bits;
                    const double mn = b == 0xffffffffffffffffull ? __longlong_as_double(0x7ff0000000000000ll)
                                                                : __longlong_as_double((long long)b);
                    if (!(dl > 0.0) || mn <= hint) s_skip = 1;
                    hint = __longlong_as_double(0x7ff0000000000000ll);
                }
                s_hint = hint;
                // the hint's threshold, set with the last step (-inf: no hint, keep every source)
                s_lnthr = hint < 1e300 ? st->lnthr[0] : -__int_as_float(0x7f800000);
            } else {
                s_lnthr = st->lnthr[OP == OP_HALF ? 1 : 2];
            }
            s_f[0] = float(h);
            s_f[1] = float(st->K1);
            s_f[2] = float(st->K3);
            s_f[3] = float(st->K4);
        }
        __syncthreads();
        if (s_skip) { __syncthreads(); continue; }
        const long long idx = base + threadIdx.x;
        const bool mine = idx < total && idx >= offsets[gi] && (gi + 1 >= ngrid || idx < offsets[gi + 1]) &&
                          idx - offsets[gi] >= G.cell_lo && idx - offsets[gi] < G.cell_hi;
        const bool stepping = s_h > 0.0;
        const bool active = mine && (OP == OP_RATEDT ? !st->done : stepping);
        double dtmin = __longlong_as_double(0x7ff0000000000000ll);
        float dtmin_f = __int_as_float(0x7f800000);
        float ions_f = 0.0f, rec_f = 0.0f;
        double ions = 0.0, rec = 0.0;
        bool defer = false;
        if (active) {
            const long long g = idx - offsets[gi];
            const int X = (int)(g % G.nx);
            const int Y = (int)((g / G.nx) % G.ny);
            const int Z = (int)(g / ((long long)G.nx * G.ny));
            const Real n = G.n ? G.n[g] : G.n_uniform;
            const Real x0 = G.x[g];
            const Real c = G.alpha * n;
            const float lnthr = s_lnthr;
            if (OP == OP_RATEDT) {
                // Eq. 4 with T fixed: K1 t_rec, K3 max(0.05, x)/|dx/dt|, K4/|dx/dt|,
                // from the sources that can matter within the hint (their bounds);
                // a cell that none of them reaches is photon-free (F = F' = 0).
                // the records of this pass: with the hint's negligible columns, or none when verifying
                const SrcSel<Real> *sel = G.sel + (verify ? 3 : 0) * MAX_SRC;
                float ampsum = 0.0f;
                Real F = Real(0), dF = Real(0);
                for (int s0 = 0; s0 < G.nsrc; s0 += 8) {
                    Real Nb[8];
                    load_columns8(G, G.N1, s0, g, Nb);
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int s = s0 + q;
                        if (s >= G.nsrc) break;
                        const Real N = Nb[q];
                        const SrcSel<Real> &S = sel[s];
                        if (N >= S.nst) continue;
                        int i, j, k;
                        const float la = sel_lnamp(S, X, Y, Z, N, i, j, k);
                        if (!(la > lnthr)) continue;
                        ampsum += __expf(la);
                        SrcRate<Real> t;
                        src_rate<Real>(t, G.qfac[s], G.tab[s], G.sigma0, G.dx, n, G.pcode[s] != 0, i, j, k, N, tabs);
                        Real Fs = Real(0), dFs = Real(0);
                        src_F_term<Real>(t, tabs, x0, Fs, dFs);       // this source's term of F(x0), F'(x0)
                        F += Fs;
                        dF += dFs;
                    }
                }
                if (rcache) {
                    rcache[idx] = F;
                    rcache[total + idx] = dF;
                    rcache[2 * total + idx] = Real(ampsum);
                }
                if (F32) {
                    if (s_f[1] > 0.0f) dtmin_f = fminf(dtmin_f, s_f[1] / (float(G.alpha) * float(n)));
                    const float xd = fabsf(float(-F + c * (Real(1) - x0) * (Real(1) - x0)));
                    if (xd > 0.0f) {
                        if (s_f[2] > 0.0f) dtmin_f = fminf(dtmin_f, s_f[2] * fmaxf(0.05f, float(x0)) / xd);
                        if (s_f[3] > 0.0f) dtmin_f = fminf(dtmin_f, s_f[3] / xd);
                    }
                } else {
                    if (st->K1 > 0) dtmin = fmin(dtmin, st->K1 / (double(G.alpha) * double(n)));
                    const double xd = fabs((double)(-F + c * (Real(1) - x0) * (Real(1) - x0)));
                    if (xd > 0) {
                        if (st->K3 > 0) dtmin = fmin(dtmin, st->K3 * fmax(0.05, (double)x0) / xd);
                        if (st->K4 > 0) dtmin = fmin(dtmin, st->K4 / xd);
                    }
                }
            } else {
                const Real h = F32 ? Real(s_f[0]) : Real(s_h);
                IntResult<Real> R;
                R.x = x0; R.IR = Real(0); R.lnfav = Real(0);
                bool done = false;
                Real F0 = Real(0), dF0 = Real(0);
                bool have_F = false;
                const bool cached = (OP == OP_HALF || OP == OP_FULL1) && use_cache && rcache;
                if (cached) {
                    const Real ampsum = rcache[2 * total + idx];
                    if (!(ampsum * h > Real(1e-3) * RealLimits<Real>::eps())) {
                        // photon-free: du/dt = -c u^2, u = 1 - x
                        const Real u0 = Real(1) - x0;
                        const Real u = u0 / (Real(1) + c * u0 * h);
                        R.x = Real(1) - u;
                        R.IR = u0 - u;
                        done = true;
                    } else {
                        F0 = rcache[idx];
                        dF0 = rcache[total + idx];
                        if (F0 == F0) {        // the dt pass formed F (not skipped)
                            have_F = true;
                            // no source's optical depth per unit x exceeds sigma0 n dx sqrt(3)
                            const Real bm = G.sigma0 * n * G.dx * Real(1.7320508075688772);
                            done = closed_form_from_F<Real>(c, x0, h, F0, dF0, bm, R);
                        }
                    }
                }
                if (!done) {
                    SrcRate<Real> r[NACT];
                    const Real *Ncol = (OP == OP_FULL2) ? G.N2 : G.N1;
                    const SrcSel<Real> *sel = G.sel + (OP == OP_HALF ? 1 : 2) * MAX_SRC;
                    const int na = gather_rates_sel<Real, NACT>(G, sel, Ncol, tabs, X, Y, Z, g, n, lnthr, r);
                    if (na <= NACT) {
                        CellODE<Real> C;
                        C.ns = na; C.c = c; C.b0 = Real(0); C.r = r; C.tabs = tabs;
                        Real f0;
                        done = integrate_prelude<Real, NACT>(C, x0, h, G.sigma0, R, F0, dF0, f0, have_F && na > 0);
                    }
                }
                if (done) {
                    if (OP == OP_HALF) {
                        const_cast<Real *>(G.xh)[g] = R.x;
                    } else {
                        G.xout[g] = R.x;
                        if (F32) {
                            ions_f = float(n) * (float(x0) - float(R.x));
                            rec_f = float(n) * float(R.IR);
                        } else {
                            const double nV = double(n) * st->cell_volume;
                            ions = nV * (double(x0) - double(R.x));
                            rec = nV * double(R.IR);
                        }
                    }
                } else {
                    defer = true;
                }
            }
        }
        if (OP != OP_RATEDT) {
            const unsigned m = __ballot_sync(0xffffffffu, defer);
            if (m) {
                const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
                unsigned qb = 0;
                if (lane == leader) qb = atomicAdd(qcount + (OP == OP_HALF ? 0 : 1), (unsigned)__popc(m));
                qb = __shfl_sync(0xffffffffu, qb, leader);
                if (defer) queue[qb + __popc(m & ((1u << lane) - 1u))] = (unsigned)idx;
            }
        }
        if (OP == OP_RATEDT) {
            if (F32) {
                for (int o = 16; o > 0; o >>= 1) dtmin_f = fminf(dtmin_f, __shfl_down_sync(0xffffffffu, dtmin_f, o));
                if ((threadIdx.x & 31) == 0) dtmin = double(dtmin_f);
            } else {
                for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_down_sync(0xffffffffu, dtmin, o));
            }
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            __syncthreads();
            if (lane == 0) sh[wid] = dtmin;
            __syncthreads();
            if (threadIdx.x == 0) {
                double mn = sh[0];
                for (int w = 1; w < (int)(blockDim.x >> 5); w++) mn = fmin(mn, sh[w]);
                // (the read skips the atomic of a block that cannot lower the minimum)
                const unsigned long long mb = (unsigned long long)__double_as_longlong(mn);
                if (mn < 1e300 && mb < *(volatile unsigned long long *)&st->dt_bits) atomicMin(&st->dt_bits, mb);
            }
        } else if (OP == OP_FULL1 || OP == OP_FULL2) {
            double si = ions, sr = rec;
            if (F32) block_sum2_f(ions_f, rec_f, st->cell_volume, si, sr, sh);
            else block_sum2(si, sr, sh);
            if (threadIdx.x == 0 && (si != 0.0 || sr != 0.0)) {
                atomicAdd(&st->bud_step[1], si + sr);
                atomicAdd(&st->bud_step[2], si);
                atomicAdd(&st->bud_step[3], sr);
            }
        }
        __syncthreads();
    }
    __syncthreads();
    }
}

// General pass of grids with several sources: one lane group per queued
// cell, as cell_general_kernel, with the sources selected for the step.
template <typename Real, int OP>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 4 : 2)
cell_multi_general_kernel(const GridDev<Real> *grids, int ngrid, const long long *offsets, const DevTable<Real> *tabs,
                          const unsigned *queue, unsigned *qcount)
{
    __shared__ double s_ions[8], s_rec[8];
    __shared__ int s_gid[8];
    constexpr int W = GroupWidth<Real>::value;
    const int lane32 = threadIdx.x & 31;
    const int gbase = lane32 & ~(W - 1), lane = lane32 - gbase;
    const unsigned gmask = W == 32 ? 0xffffffffu : (0xffffu << gbase);
    if (OP != OP_HALF) {
        if (threadIdx.x < 8) { s_ions[threadIdx.x] = 0.0; s_rec[threadIdx.x] = 0.0; s_gid[threadIdx.x] = -1; }
        __syncthreads();
    }
    const int qi = OP == OP_HALF ? 0 : 1;
    const unsigned nq = qcount[qi];
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(&qcount[2 + qi], 1u);
        q = __shfl_sync(gmask, q, gbase);
        if (q >= nq) break;
        const long long idx = queue[q];
        const int gi = find_grid(offsets, ngrid, idx);
        const GridDev<Real> &G = grids[gi];
        DevState *st = G.st;
        const double dtd = st->dt;
        const long long g = idx - offsets[gi];
        const int X = (int)(g % G.nx);
        const int Y = (int)((g / G.nx) % G.ny);
        const int Z = (int)(g / ((long long)G.nx * G.ny));
        const Real n = G.n ? G.n[g] : G.n_uniform;
        const Real x0 = G.x[g];
        const Real *Ncol = (OP == OP_FULL2) ? G.N2 : G.N1;
        const double hd = OP == OP_HALF ? 0.5 * dtd : dtd;
        const Real h = Real(hd);
        const float lnthr = st->lnthr[OP == OP_HALF ? 1 : 2];
        IntResult<Real> R;
        Real F0, dF0, f0;
        // the sources selected for the step (as the closed-form pass selected them),
        // in local memory; one instantiation of the integrator keeps the kernel's
        // code small (its lanes run apart through the root search and quadrature)
        SrcRate<Real> ra[MAX_SRC];
        const SrcSel<Real> *sel = G.sel + (OP == OP_HALF ? 1 : 2) * MAX_SRC;
        CellODE<Real> C;
        C.ns = gather_rates_sel<Real, MAX_SRC>(G, sel, Ncol, tabs, X, Y, Z, g, n, lnthr, ra);
        C.c = G.alpha * n; C.b0 = Real(0); C.r = ra; C.tabs = tabs;
        if (!integrate_prelude<Real, MAX_SRC>(C, x0, h, G.sigma0, R, F0, dF0, f0))
            R = integrate_general<Real, MAX_SRC>(C, x0, h, G.sigma0, R, F0, dF0, f0, GroupEval<W>{lane, gbase, gmask});
        if (lane == 0) {
            if (OP == OP_HALF) {
                const_cast<Real *>(G.xh)[g] = R.x;
            } else {
                G.xout[g] = R.x;
                const double nV = double(n) * st->cell_volume;
                const double ions = nV * (double(x0) - double(R.x)), rec = nV * double(R.IR);
                const int slot = gi & 7;
                const int owner = atomicCAS(&s_gid[slot], -1, gi);
                if (owner == -1 || owner == gi) {
                    atomicAdd(&s_ions[slot], ions);
                    atomicAdd(&s_rec[slot], rec);
                } else {
                    atomicAdd(&st->bud_step[1], ions + rec);
                    atomicAdd(&st->bud_step[2], ions);
                    atomicAdd(&st->bud_step[3], rec);
                }
            }
        }
    }
    if (OP != OP_HALF) {
        __syncthreads();
        if (threadIdx.x < 8 && s_gid[threadIdx.x] >= 0) {
            DevState *st = grids[s_gid[threadIdx.x]].st;
            atomicAdd(&st->bud_step[1], s_ions[threadIdx.x] + s_rec[threadIdx.x]);
            atomicAdd(&st->bud_step[2], s_ions[threadIdx.x]);
            atomicAdd(&st->bud_step[3], s_rec[threadIdx.x]);
        }
    }
}

// stage 0: choose dt (Eq. 4 minimum or fixed, capped at t_end - t) and reset the step budget
// stage 1: close the substep (t += dt, totals, done flag)
template <typename Real>
__global__ void finalize_kernel(const GridDev<Real> *grids, int ngrid, int stage, unsigned *qcount,
                                const DevTable<Real> *tabs)
{
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (stage == 0 && gi == 0) { qcount[0] = 0u; qcount[1] = 0u; qcount[2] = 0u; qcount[3] = 0u; }
    if (gi >= ngrid) return;
    DevState *st = grids[gi].st;
    if (stage == 0) {
        double dt = 0.0, dcrit = 0.0;
        if (!st->done) {
            if (st->dt_fixed > 0) dt = st->dt_fixed;
            else if (st->dt_bits != 0xffffffffffffffffull) dt = __longlong_as_double((long long)st->dt_bits);
            else dt = st->t_end - st->t;
            dcrit = dt;
            const double rem = st->t_end - st->t;
            if (dt >= rem * (1.0 - 1e-12)) dt = rem;
            if (!(dt > 0.0)) { dt = 0.0; st->done = 1; }
        }
        st->dt = dt;
        // the hint of the next dt pass: the step the criterion asked for (a
        // step cut short to land on t_end leaves it as it was asked)
        if (dt > 0.0) {
            st->dt_last = dcrit > dt ? dcrit : dt;
            st->lnthr[0] = lnthr_step<Real>(4.0 * st->dt_last);
            st->lnthr[1] = lnthr_step<Real>(0.5 * dt);
            st->lnthr[2] = lnthr_step<Real>(dt);
        }
        st->dt_bits = 0xffffffffffffffffull;
        const GridDev<Real> &G = grids[gi];
        if (G.sel && dt > 0.0) {
            // negligible columns of the next dt pass (its hint, 4 dt_last), the half step and the full step
            for (int s = 0; s < G.nsrc; s++) {
                G.sel[s].nst = negligible_column<Real>(G, tabs, s, st->lnthr[0]);
                G.sel[MAX_SRC + s].nst = negligible_column<Real>(G, tabs, s, st->lnthr[1]);
                G.sel[2 * MAX_SRC + s].nst = negligible_column<Real>(G, tabs, s, st->lnthr[2]);
            }
        }
        st->bud_step[0] = st->sumQ * dt;
        st->bud_step[1] = st->bud_step[2] = st->bud_step[3] = 0.0;
    } else {
        if (st->dt > 0.0) {
            st->t += st->dt;
            st->nsub += 1;
            for (int q = 0; q < 4; q++) st->bud_total[q] += st->bud_step[q];
            if (st->t >= st->t_end) st->done = 1;
        }
    }
}

template <typename Real, int NSMAX, int BS>
static cudaError_t launch_cell_ns(const GridDev<Real> *grids, int ngrid, const long long *offsets, long long total,
                                  const DevTable<Real> *tabs, int op, unsigned *queue, unsigned *qcount,
                                  Real *qrec, Real *rcache, int use_cache, int gen_blocks, cudaStream_t s)
{
    const long long nb = (total + BS - 1) / BS;
    const int gbs = 256;                 // the general pass's blocks
    switch (op) {
    case OP_RATEDT: cell_kernel<Real, OP_RATEDT, NSMAX, BS><<<(unsigned)nb, BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, qrec, rcache, use_cache); break;
    case OP_HALF: cell_kernel<Real, OP_HALF, NSMAX, BS><<<(unsigned)nb, BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, qrec, rcache, use_cache); break;
    case OP_FULL1: cell_kernel<Real, OP_FULL1, NSMAX, BS><<<(unsigned)nb, BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, qrec, rcache, use_cache); break;
    case OP_FULL2: cell_kernel<Real, OP_FULL2, NSMAX, BS><<<(unsigned)nb, BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, qrec, rcache, use_cache); break;
    case OP_HALF | OP_GENERAL: cell_general_kernel<Real, OP_HALF, NSMAX><<<gen_blocks, gbs, 0, s>>>(grids, ngrid, offsets, tabs, queue, qcount, qrec); break;
    case OP_FULL1 | OP_GENERAL: cell_general_kernel<Real, OP_FULL1, NSMAX><<<gen_blocks, gbs, 0, s>>>(grids, ngrid, offsets, tabs, queue, qcount, qrec); break;
    case OP_FULL2 | OP_GENERAL: cell_general_kernel<Real, OP_FULL2, NSMAX><<<gen_blocks, gbs, 0, s>>>(grids, ngrid, offsets, tabs, queue, qcount, qrec); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename Real, int BS>
static cudaError_t launch_cell_multi(const GridDev<Real> *grids, int ngrid, const long long *offsets, long long total,
                                     const DevTable<Real> *tabs, int op, unsigned *queue, unsigned *qcount,
                                     Real *rcache, int uc, int gen_blocks, cudaStream_t s)
{
    const long long nb = (total + BS - 1) / BS;
    const int gbs = 256;                 // the general pass's blocks
    switch (op) {
    case OP_RATEDT:
        cell_multi_kernel<Real, OP_RATEDT, BS><<<(unsigned)nb, BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, rcache, uc, 0);
        break;
    case OP_RATEDT_VERIFY:
        // the verifying pass: a few resident blocks that return unless the minimum exceeded the hint
        cell_multi_kernel<Real, OP_RATEDT, BS><<<(unsigned)std::min<long long>(nb, 8LL * gen_blocks * (256 / BS)), BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, rcache, uc, 1);
        break;
    case OP_HALF: cell_multi_kernel<Real, OP_HALF, BS><<<(unsigned)nb, BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, rcache, uc, 0); break;
    case OP_FULL1: cell_multi_kernel<Real, OP_FULL1, BS><<<(unsigned)nb, BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, rcache, uc, 0); break;
    case OP_FULL2: cell_multi_kernel<Real, OP_FULL2, BS><<<(unsigned)nb, BS, 0, s>>>(grids, ngrid, offsets, total, tabs, queue, qcount, rcache, uc, 0); break;
    case OP_HALF | OP_GENERAL: cell_multi_general_kernel<Real, OP_HALF><<<gen_blocks, gbs, 0, s>>>(grids, ngrid, offsets, tabs, queue, qcount); break;
    case OP_FULL1 | OP_GENERAL: cell_multi_general_kernel<Real, OP_FULL1><<<gen_blocks, gbs, 0, s>>>(grids, ngrid, offsets, tabs, queue, qcount); break;
    case OP_FULL2 | OP_GENERAL: cell_multi_general_kernel<Real, OP_FULL2><<<gen_blocks, gbs, 0, s>>>(grids, ngrid, offsets, tabs, queue, qcount); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// nsmax: the largest source count of the grids in the call (1 selects the
// single-source kernels, whose per-source state stays in registers).  cell_bs:
// threads per block of the closed-form passes (256; anything else: 128).
template <typename Real>
cudaError_t launch_cell(const GridDev<Real> *grids, int ngrid, const long long *offsets, long long total,
                        const DevTable<Real> *tabs, int op, int nsmax, unsigned *queue, unsigned *qcount,
                        Real *qrec, Real *rcache, int use_cache, int gen_blocks, int cell_bs, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    if (op == OP_RATEDT_VERIFY && nsmax <= 1) return cudaSuccess;     // the single-source pass uses no hint
    const int uc = use_cache && rcache ? 1 : 0;
    if (nsmax <= 1)
        return cell_bs == 256
                   ? launch_cell_ns<Real, 1, 256>(grids, ngrid, offsets, total, tabs, op, queue, qcount, qrec, rcache, uc, gen_blocks, s)
                   : launch_cell_ns<Real, 1, 128>(grids, ngrid, offsets, total, tabs, op, queue, qcount, qrec, rcache, uc, gen_blocks, s);
    return cell_bs == 256
               ? launch_cell_multi<Real, 256>(grids, ngrid, offsets, total, tabs, op, queue, qcount, rcache, uc, gen_blocks, s)
               : launch_cell_multi<Real, 128>(grids, ngrid, offsets, total, tabs, op, queue, qcount, rcache, uc, gen_blocks, s);
}

template <typename Real> size_t queue_record_bytes() { return QREC * sizeof(Real); }

// Resident 256-thread blocks of the general pass per SM.
template <typename Real>
int cell_general_occupancy(int nsmax)
{
    int nb = 0;
    cudaError_t e = nsmax <= 1
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_general_kernel<Real, OP_FULL2, 1>, 256, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cell_multi_general_kernel<Real, OP_FULL2>, 256, 0);
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

template <typename Real>
cudaError_t launch_finalize(const GridDev<Real> *grids, int ngrid, int stage, unsigned *qcount,
                            const DevTable<Real> *tabs, cudaStream_t s)
{
    finalize_kernel<Real><<<(ngrid + 63) / 64, 64, 0, s>>>(grids, ngrid, stage, qcount, tabs);
    return cudaGetLastError();
}

template cudaError_t launch_cell<double>(const GridDev<double> *, int, const long long *, long long,
                                         const DevTable<double> *, int, int, unsigned *, unsigned *, double *, double *,
                                         int, int, int, cudaStream_t);
template cudaError_t launch_cell<float>(const GridDev<float> *, int, const long long *, long long,
                                        const DevTable<float> *, int, int, unsigned *, unsigned *, float *, float *, int,
                                        int, int, cudaStream_t);
template size_t queue_record_bytes<double>();
template size_t queue_record_bytes<float>();
template int cell_general_occupancy<double>(int);
template int cell_general_occupancy<float>(int);
template cudaError_t launch_finalize<double>(const GridDev<double> *, int, int, unsigned *, const DevTable<double> *,
                                             cudaStream_t);
template cudaError_t launch_finalize<float>(const GridDev<float> *, int, int, unsigned *, const DevTable<float> *,
                                            cudaStream_t);

} // namespace oots
