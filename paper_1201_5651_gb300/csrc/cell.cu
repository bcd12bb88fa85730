// Per-cell passes of a substep (Mackey 2012, Sect. 2.2): the timestep
// criterion of Eq. 4 (minimum over all cells), the half-step and full-step
// integrations of Eq. 2 with frozen entry columns, and the photon budget.
// Elementwise over every cell of every grid of the call; one flat index space,
// grids located by binary search over their cell offsets.
#include "common.cuh"
#include "integrator.cuh"
#include "kernels.h"

namespace oots {

__device__ __forceinline__ int find_grid(const long long *off, int ngrid, long long idx)
{
    int lo = 0, hi = ngrid - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Rate parameters of every source for the cell at global index g = (X,Y,Z).
template <typename Real, int NSMAX>
__device__ __forceinline__ int cell_rates(const GridDev<Real> &G, const Real *Ncol, const DevTable<Real> *tabs,
                                          int X, int Y, int Z, long long g, Real n, SrcRate<Real> *r)
{
    for (int s = 0; s < NSMAX && s < G.nsrc; s++) {
        const int i = X >= G.vtx[s][0] ? X - G.vtx[s][0] : G.vtx[s][0] - 1 - X;
        const int j = Y >= G.vtx[s][1] ? Y - G.vtx[s][1] : G.vtx[s][1] - 1 - Y;
        const int k = Z >= G.vtx[s][2] ? Z - G.vtx[s][2] : G.vtx[s][2] - 1 - Z;
        const Real c0 = Real(i) + Real(0.5), c1 = Real(j) + Real(0.5), c2 = Real(k) + Real(0.5);
        const Real r2 = c0 * c0 + c1 * c1 + c2 * c2;
        const Real sf = m_sqrt(r2) / m_max(c0, m_max(c1, c2));
        const Real N = Ncol[(long long)s * G.ncell + g];
        r[s].Nin = N;
        r[s].tab = G.tab[s];
        if (r[s].tab < 0) {
            // Q e^{-sigma0 N} / (n 4 pi r^2 ds) with r^2 ds in units of dx^3
            r[s].A = G.qfac[s] * m_exp(-G.sigma0 * N) / (n * r2 * sf);
            r[s].b = G.sigma0 * n * G.dx * sf;
            r[s].p = Real(1);
        } else {
            r[s].A = G.qfac[s] / (n * r2 * sf);
            r[s].b = n * G.dx * sf;
            r[s].p = m_exp(tab_lnp(tabs[r[s].tab], N));
        }
    }
    return G.nsrc;
}

template <typename Real>
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
    return s;
}

template <typename Real, int OP, int NSMAX>
__global__ void __launch_bounds__(256) cell_kernel(const GridDev<Real> *grids, int ngrid, const long long *offsets,
                                                   long long total, const DevTable<Real> *tabs)
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
    }
    __syncthreads();
    for (int gi = s_grid_lo; gi <= s_grid_hi; gi++) {
        const GridDev<Real> &G = grids[gi];
        DevState *st = G.st;
        const long long idx = base + threadIdx.x;
        const bool mine = idx < total && idx >= offsets[gi] && (gi + 1 >= ngrid || idx < offsets[gi + 1]);
        const double dtd = st->dt;
        const bool active = mine && (OP == OP_RATEDT || dtd > 0.0) && !(OP == OP_RATEDT && st->done);
        double dtmin = __longlong_as_double(0x7ff0000000000000ll);
        double ions = 0.0, rec = 0.0;
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
            C.ns = cell_rates<Real, NSMAX>(G, Ncol, tabs, X, Y, Z, g, n, r);
            C.c = G.alpha * n;
            C.b0 = Real(0);
            C.r = r;
            C.tabs = tabs;
            if (OP == OP_RATEDT) {
                // Eq. 4 with T fixed: K1 t_rec, K3 max(0.05, x)/|dx/dt|, K4/|dx/dt|
                const double xd = fabs((double)ode_rhs<Real, NSMAX>(C, x0));
                if (st->K1 > 0) dtmin = fmin(dtmin, st->K1 / (double(G.alpha) * double(n)));
                if (xd > 0) {
                    if (st->K3 > 0) dtmin = fmin(dtmin, st->K3 * fmax(0.05, (double)x0) / xd);
                    if (st->K4 > 0) dtmin = fmin(dtmin, st->K4 / xd);
                }
            } else if (OP == OP_HALF) {
                IntResult<Real> R = integrate_cell<Real, NSMAX>(C, x0, Real(0.5 * dtd), G.sigma0);
                const_cast<Real *>(G.xh)[g] = R.x;
            } else {
                IntResult<Real> R = integrate_cell<Real, NSMAX>(C, x0, Real(dtd), G.sigma0);
                G.xout[g] = R.x;
                const double nV = double(n) * st->cell_volume;
                ions = nV * (double(x0) - double(R.x));
                rec = nV * double(R.IR);
            }
        }
        if (OP == OP_RATEDT) {
            for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_down_sync(0xffffffffu, dtmin, o));
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            __syncthreads();
            if (lane == 0) sh[wid] = dtmin;
            __syncthreads();
            if (threadIdx.x == 0) {
                double m = sh[0];
                for (int w = 1; w < (int)(blockDim.x >> 5); w++) m = fmin(m, sh[w]);
                if (m < 1e300) atomicMin(&st->dt_bits, (unsigned long long)__double_as_longlong(m));
            }
        } else if (OP == OP_FULL1 || OP == OP_FULL2) {
            const double si = block_sum<Real>(ions, sh);
            const double sr = block_sum<Real>(rec, sh);
            if (threadIdx.x == 0 && (si != 0.0 || sr != 0.0)) {
                atomicAdd(&st->bud_step[1], si + sr);   // absorbed = new ions + recombinations
                atomicAdd(&st->bud_step[2], si);
                atomicAdd(&st->bud_step[3], sr);
            }
        }
        __syncthreads();
    }
}

// stage 0: choose dt (Eq. 4 minimum or fixed, capped at t_end - t) and reset the step budget
// stage 1: close the substep (t += dt, totals, done flag)
template <typename Real>
__global__ void finalize_kernel(const GridDev<Real> *grids, int ngrid, int stage)
{
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ngrid) return;
    DevState *st = grids[gi].st;
    if (stage == 0) {
        double dt = 0.0;
        if (!st->done) {
            if (st->dt_fixed > 0) dt = st->dt_fixed;
            else if (st->dt_bits != 0xffffffffffffffffull) dt = __longlong_as_double((long long)st->dt_bits);
            else dt = st->t_end - st->t;
            const double rem = st->t_end - st->t;
            if (dt >= rem * (1.0 - 1e-12)) dt = rem;
            if (!(dt > 0.0)) { dt = 0.0; st->done = 1; }
        }
        st->dt = dt;
        st->dt_bits = 0xffffffffffffffffull;
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

template <typename Real, int NSMAX>
static cudaError_t launch_cell_ns(const GridDev<Real> *grids, int ngrid, const long long *offsets, long long total,
                                  const DevTable<Real> *tabs, int op, cudaStream_t s)
{
    const int bs = 256;
    const long long nb = (total + bs - 1) / bs;
    switch (op) {
    case OP_RATEDT: cell_kernel<Real, OP_RATEDT, NSMAX><<<(unsigned)nb, bs, 0, s>>>(grids, ngrid, offsets, total, tabs); break;
    case OP_HALF: cell_kernel<Real, OP_HALF, NSMAX><<<(unsigned)nb, bs, 0, s>>>(grids, ngrid, offsets, total, tabs); break;
    case OP_FULL1: cell_kernel<Real, OP_FULL1, NSMAX><<<(unsigned)nb, bs, 0, s>>>(grids, ngrid, offsets, total, tabs); break;
    case OP_FULL2: cell_kernel<Real, OP_FULL2, NSMAX><<<(unsigned)nb, bs, 0, s>>>(grids, ngrid, offsets, total, tabs); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// nsmax: the largest source count of the grids in the call (1 selects the
// single-source kernels, whose per-source state stays in registers)
template <typename Real>
cudaError_t launch_cell(const GridDev<Real> *grids, int ngrid, const long long *offsets, long long total,
                        const DevTable<Real> *tabs, int op, int nsmax, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    if (nsmax <= 1) return launch_cell_ns<Real, 1>(grids, ngrid, offsets, total, tabs, op, s);
    return launch_cell_ns<Real, MAX_SRC>(grids, ngrid, offsets, total, tabs, op, s);
}

template <typename Real>
cudaError_t launch_finalize(const GridDev<Real> *grids, int ngrid, int stage, cudaStream_t s)
{
    finalize_kernel<Real><<<(ngrid + 63) / 64, 64, 0, s>>>(grids, ngrid, stage);
    return cudaGetLastError();
}

template cudaError_t launch_cell<double>(const GridDev<double> *, int, const long long *, long long,
                                         const DevTable<double> *, int, int, cudaStream_t);
template cudaError_t launch_cell<float>(const GridDev<float> *, int, const long long *, long long,
                                        const DevTable<float> *, int, int, cudaStream_t);
template cudaError_t launch_finalize<double>(const GridDev<double> *, int, int, cudaStream_t);
template cudaError_t launch_finalize<float>(const GridDev<float> *, int, int, cudaStream_t);

} // namespace oots
