// Plane-parallel sources: a source at infinity whose rays run along a grid
// axis (the slab test of Mackey 2012, Sect. 3.1).  With parallel rays the
// short-characteristics interpolation reduces to the one upwind cell on the
// same row, so the column to the entry of a cell is the sum of n x dx over the
// cells before it on its row and every row is independent:
//   - trace: an exclusive prefix sum of n x dx along each row (FP64 sums in
//     both precisions), written to the source's column array;
//   - implicit (A1, Sect. 2.1, Eq. 3): along each row, in the direction of
//     travel, every cell is integrated over dt with its entry column frozen and
//     hands downstream N_out = N_in - ln<f>/sigma0 from its time-averaged
//     attenuation <f>.
// The rate of a cell (Sect. 2 photon-conserving form) shares the photons the
// row loses in it over the cell volume per unit face area, dx (src_rate with
// plane = true).
//
// Row layout (x fastest): rows of axis 0 are contiguous and take one warp each
// (a warp scan over 32 cells at a time); rows of axes 1 and 2 take one thread
// each, numbered so that neighbouring threads hold neighbouring x and every
// load of a warp is one coalesced line.
#include "common.cuh"
#include "integrator.cuh"
#include "kernels.h"

namespace oots {

struct PlaneRow {
    long long base;    // first cell on the direction of travel
    long long step;    // index step to the next cell downstream (negative for back = 1)
    int len;           // cells on the row
};

template <typename Real>
__device__ __forceinline__ PlaneRow plane_row(const GridDev<Real> &G, int code, long long r)
{
    const int axis = code >> 1, back = code & 1;
    const long long nxy = (long long)G.nx * G.ny;
    PlaneRow R;
    if (axis == 0) {                 // r = Y + ny Z
        R.base = r * G.nx; R.step = 1; R.len = G.nx;
    } else if (axis == 1) {          // r = X + nx Z
        const long long X = r % G.nx, Z = r / G.nx;
        R.base = X + nxy * Z; R.step = G.nx; R.len = G.ny;
    } else {                         // r = X + nx Y
        R.base = r; R.step = nxy; R.len = G.nz;
    }
    if (back) { R.base += (long long)(R.len - 1) * R.step; R.step = -R.step; }
    return R;
}

__device__ __forceinline__ int find_plane_job(const PlaneJob *jobs, int njobs, long long t)
{
    int j = 0;
    while (j + 1 < njobs && jobs[j + 1].first <= t) j++;
    return j;
}

template <typename Real>
__device__ __forceinline__ Real cell_n(const GridDev<Real> &G, long long g)
{
    return G.n ? __ldg(G.n + g) : G.n_uniform;
}

// Columns of every plane source of the launch: which = 0 traces x into N1,
// which = 1 traces the half-step state xh into N2.
template <typename Real>
__global__ void __launch_bounds__(256) plane_trace_kernel(const GridDev<Real> *grids, const PlaneJob *jobs, int njobs,
                                                          long long nthreads, int which)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t - (threadIdx.x & 31) >= nthreads) return;           // whole warps leave together
    const PlaneJob J = jobs[find_plane_job(jobs, njobs, t - (threadIdx.x & 31))];
    const GridDev<Real> &G = grids[J.grid];
    const Real *x = which ? G.xh : G.x;
    Real *Nout = (which ? G.N2 : G.N1) + (long long)J.src * G.ncell;
    const double dx = double(G.dx);
    if ((J.code >> 1) == 0) {
        // one warp per row: exclusive warp scans, 32 cells at a time
        const long long r = (t - J.first) >> 5;
        if (r >= J.rows) return;                                 // uniform over the warp
        const int lane = threadIdx.x & 31;
        const PlaneRow R = plane_row(G, J.code, r);
        double carry = 0.0;
        for (int m0 = 0; m0 < R.len; m0 += 32) {
            const int m = m0 + lane;
            const long long g = R.base + (long long)m * R.step;
            double dN = 0.0;
            if (m < R.len) dN = double(cell_n(G, g)) * double(x[g]) * dx;
            double inc = dN;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            double exc = __shfl_up_sync(0xffffffffu, inc, 1);
            if (lane == 0) exc = 0.0;
            if (m < R.len) Nout[g] = Real(carry + exc);
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        return;
    }
    // one thread per row; loads of a block of cells are issued before the stores
    const long long r = t - J.first;
    if (r >= J.rows) return;
    const PlaneRow R = plane_row(G, J.code, r);
    constexpr int B = 8;
    double N = 0.0;
    for (int m0 = 0; m0 < R.len; m0 += B) {
        double dN[B];
#pragma unroll
        for (int q = 0; q < B; q++) {
            const long long g = R.base + (long long)(m0 + q) * R.step;
            dN[q] = (m0 + q < R.len) ? double(cell_n(G, g)) * double(x[g]) * dx : 0.0;
        }
#pragma unroll
        for (int q = 0; q < B; q++) {
            if (m0 + q < R.len) Nout[R.base + (long long)(m0 + q) * R.step] = Real(N);
            N += dN[q];
        }
    }
}

// A1 with a plane source: one thread per row integrates its cells in the
// direction of travel; photon budget by warp sums, one atomic per warp.
template <typename Real>
__global__ void __launch_bounds__(128) plane_implicit_kernel(const GridDev<Real> *grids, const PlaneJob *jobs,
                                                             int njobs, long long nthreads,
                                                             const DevTable<Real> *tabs)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t - (threadIdx.x & 31) >= nthreads) return;
    const PlaneJob J = jobs[find_plane_job(jobs, njobs, t - (threadIdx.x & 31))];
    const GridDev<Real> &G = grids[J.grid];
    const long long r = t - J.first;
    double ions = 0.0, rec = 0.0;
    const Real dt = Real(G.st->dt);
    if (r < J.rows) {
        const PlaneRow R = plane_row(G, J.code, r);
        const int s = J.src;
        const Real sig = G.sigma0;
        const double cellV = G.st->cell_volume;
        Real *N1 = G.N1 + (long long)s * G.ncell;
        double N = 0.0;
        for (int m = 0; m < R.len; m++) {
            const long long g = R.base + (long long)m * R.step;
            const Real n = cell_n(G, g);
            const Real x0 = G.x[g];
            SrcRate<Real> rt;
            src_rate<Real>(rt, G.qfac[s], G.tab[s], sig, G.dx, n, true, 0, 0, 0, Real(N), tabs);
            CellODE<Real> C;
            C.ns = 1; C.c = G.alpha * n; C.b0 = sig * n * G.dx; C.r = &rt; C.tabs = tabs;
            const IntResult<Real> Rs = integrate_cell<Real, 1>(C, x0, dt, sig);
            Real dtau_eff = -Rs.lnfav;
            if (!(dtau_eff >= Real(0))) dtau_eff = Real(0);
            N1[g] = Real(N);
            N += double(dtau_eff) / double(sig);
            if (dt > Real(0)) {
                G.xout[g] = Rs.x;
                const double nV = double(n) * cellV;
                ions += nV * double(x0 - Rs.x);
                rec += nV * double(Rs.IR);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ions += __shfl_down_sync(0xffffffffu, ions, o);
        rec += __shfl_down_sync(0xffffffffu, rec, o);
    }
    if ((threadIdx.x & 31) == 0 && (ions != 0.0 || rec != 0.0)) {
        DevState *st = G.st;
        atomicAdd(&st->bud_step[2], ions);
        atomicAdd(&st->bud_step[3], rec);
        atomicAdd(&st->bud_step[1], ions + rec);
    }
}

long long plane_job_threads(int code, long long rows)
{
    const long long t = (code >> 1) == 0 ? rows * 32 : rows;
    return (t + 31) / 32 * 32;
}

template <typename Real>
cudaError_t launch_plane(const GridDev<Real> *grids, const PlaneJob *jobs, int njobs, long long nthreads,
                         const DevTable<Real> *tabs, int which, int implicit, cudaStream_t s)
{
    if (njobs <= 0 || nthreads <= 0) return cudaSuccess;
    if (implicit) {
        const int bs = 128;
        plane_implicit_kernel<Real><<<(unsigned)((nthreads + bs - 1) / bs), bs, 0, s>>>(grids, jobs, njobs, nthreads,
                                                                                        tabs);
    } else {
        const int bs = 256;
        plane_trace_kernel<Real><<<(unsigned)((nthreads + bs - 1) / bs), bs, 0, s>>>(grids, jobs, njobs, nthreads,
                                                                                     which);
    }
    return cudaGetLastError();
}

template cudaError_t launch_plane<double>(const GridDev<double> *, const PlaneJob *, int, long long,
                                          const DevTable<double> *, int, int, cudaStream_t);
template cudaError_t launch_plane<float>(const GridDev<float> *, const PlaneJob *, int, long long,
                                         const DevTable<float> *, int, int, cudaStream_t);

} // namespace oots
