// Plane-parallel sources: a source at infinity whose rays run along a grid
// axis (the slab test of Mackey 2012, Sect. 3.1).  With parallel rays the
// short-characteristics interpolation reduces to the one upwind cell on the
// same row, so the column to the entry of a cell is the sum of n x dx over the
// cells before it on its row and every row is independent:
//   - trace: an exclusive prefix sum of n x dx along each row (float-float
//     sums in the mixed path, double in the FP64 path), written to the
//     source's column array;
//   - implicit (A1, Sect. 2.1, Eq. 3): along each row, in the direction of
//     travel, every cell is integrated over dt with its entry column frozen and
//     hands downstream N_out = N_in - ln<f>/sigma0 from its time-averaged
//     attenuation <f>.
// The rate of a cell (Sect. 2 photon-conserving form) shares the photons the
// row loses in it over the cell volume per unit face area, dx (src_rate with
// plane = true).
//
// Row layout (x fastest): rows of axis 0 are contiguous and take one warp each;
// rows of axes 1 and 2 are numbered so that neighbouring rows start at
// neighbouring x, and a warp's lanes hold 32 of them, so every load of a warp
// is one coalesced line.  The trace keeps many loads in flight per thread
// (see the kernel); the A1 row integration is ALU-bound and takes one thread
// per row.
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

// Column accumulation without FP64 arithmetic in the mixed path (GB300 runs
// FP64 at a small fraction of its FP32 rate): the running sum of n x is a
// float-float (ff) value there and a double in the FP64 path, and dx is
// applied once per output.  In FP64 each cell costs two fused multiply-adds.
__device__ __forceinline__ double acc_nx(double pre, double n, double x) { return fma(n, x, pre); }
__device__ __forceinline__ ff acc_nx(ff pre, float n, float x) { return ff_add_f(pre, n * x); }
__device__ __forceinline__ double col_out(double base_dx, double pre, double dx) { return fma(pre, dx, base_dx); }
__device__ __forceinline__ float col_out(ff base, ff pre, float dx) { ff s = ff_add(base, pre); return (s.hi + s.lo) * dx; }
__device__ __forceinline__ double col_base(double base, double dx) { return base * dx; }
__device__ __forceinline__ ff col_base(ff base, float) { return base; }
__device__ __forceinline__ double shfl_up_col(double v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ ff shfl_up_col(ff v, int o)
{
    return ff{__shfl_up_sync(0xffffffffu, v.hi, o), __shfl_up_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double shfl_col(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ ff shfl_col(ff v, int l)
{
    return ff{__shfl_sync(0xffffffffu, v.hi, l), __shfl_sync(0xffffffffu, v.lo, l)};
}

// Columns of the plane sources of one launch: which = 0 traces x into N1,
// which = 1 traces the half-step state xh into N2.  Blocks of 256 threads; a
// block belongs to one job (jobs start on multiples of 256 threads); t_base is
// the launch's first thread in the jobs' numbering.  In both layouts a thread
// sums a run of consecutive cells of its row on its own and only the run
// totals are scanned across threads.
//   rows along x (ROWX): one warp per row, 256 cells at a time; lane l takes
//     cells [8l, 8l + 8) of the stretch, the 32 lane totals are scanned by
//     shuffles;
//   rows along y or z: a block holds 32 neighbouring rows (lane = row,
//     neighbouring x, so each warp load is one line) and walks them 256 cells
//     at a time; warp w takes cells [32w, 32w + 32) of the stretch, the eight
//     warp totals are scanned through shared memory.  The mixed path keeps the
//     run's products n x in registers (its loads all issue before the sums);
//     the FP64 path keeps the run's prefix sums (one fused multiply-add each).
constexpr int kRun0 = 8;     // cells per lane and stretch, rows along x
constexpr int kRun1 = 32;    // cells per lane and stretch, rows along y or z

template <typename Real, bool ROWX>
__global__ void __launch_bounds__(256, ROWX ? 3 : 2) plane_trace_kernel(const GridDev<Real> *grids,
                                                                        const PlaneJob *jobs, int njobs,
                                                                        long long t_base, long long t_end, int which)
{
    typedef typename ColT<Real>::type Col;
    const long long t0 = t_base + (long long)blockIdx.x * blockDim.x;   // first thread of the block
    if (t0 >= t_end) return;                                          // whole blocks leave together
    const PlaneJob J = jobs[find_plane_job(jobs, njobs, t0)];
    const GridDev<Real> &G = grids[J.grid];
    const Real *__restrict__ x = which ? G.xh : G.x;
    // loads without branches, so that a run's loads all issue before its sums:
    // a uniform density is read through a zero stride from the grid record,
    // and cells past the row end read the row's first cell and count zero
    const Real *__restrict__ nd = G.n ? G.n : &grids[J.grid].n_uniform;
    const long long nmul = G.n ? 1 : 0;
    Real *__restrict__ Nout = (which ? G.N2 : G.N1) + (long long)J.src * G.ncell;
    const Real dx = G.dx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (ROWX) {
        const long long r = (t0 - J.first + threadIdx.x) >> 5;
        if (r >= J.rows) return;                                   // uniform over the warp
        const PlaneRow R = plane_row(G, J.code, r);
        Col carry = ColT<Real>::zero();
        for (int m0 = 0; m0 < R.len; m0 += 32 * kRun0) {
            const int mb = m0 + kRun0 * lane;
            Real nn[kRun0], xx[kRun0];
#pragma unroll
            for (int q = 0; q < kRun0; q++) {
                const int m = mb + q;
                const long long g = R.base + (long long)(m < R.len ? m : 0) * R.step;
                const Real xv = __ldg(x + g);
                nn[q] = __ldg(nd + g * nmul);
                xx[q] = m < R.len ? xv : Real(0);
            }
            Col pre[kRun0 + 1];
            pre[0] = ColT<Real>::zero();
#pragma unroll
            for (int q = 0; q < kRun0; q++) pre[q + 1] = acc_nx(pre[q], nn[q], xx[q]);
            // exclusive scan of the lane totals
            Col inc = pre[kRun0];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const Col v = shfl_up_col(inc, o);
                if (lane >= o) inc = ColT<Real>::addc(inc, v);
            }
            Col exc = shfl_up_col(inc, 1);
            if (lane == 0) exc = ColT<Real>::zero();
            const auto base = col_base(ColT<Real>::addc(carry, exc), dx);
#pragma unroll
            for (int q = 0; q < kRun0; q++) {
                const int m = mb + q;
                if (m < R.len) Nout[R.base + (long long)m * R.step] = Real(col_out(base, pre[q], dx));
            }
            carry = ColT<Real>::addc(carry, shfl_col(inc, 31));
        }
        return;
    }
    __shared__ Col s_sum[8][33];
    __shared__ Col s_carry[32];
    const long long r = ((t0 - J.first) >> 3) + lane;              // 256 threads per 32 rows
    const bool live = r < J.rows;
    const PlaneRow R = plane_row(G, J.code, live ? r : 0);
    if (warp == 0) s_carry[lane] = ColT<Real>::zero();
    for (int m0 = 0; m0 < R.len; m0 += 8 * kRun1) {
        const int mb = m0 + kRun1 * warp;
        if (sizeof(Real) == 4) {
            Real nxp[kRun1];
#pragma unroll
            for (int q = 0; q < kRun1; q++) {
                const int m = mb + q;
                const bool in = live && m < R.len;
                const long long g = R.base + (long long)(in ? m : 0) * R.step;
                const Real xv = __ldg(x + g), nv = __ldg(nd + g * nmul);
                nxp[q] = in ? nv * xv : Real(0);
            }
            Col tot = ColT<Real>::zero();
#pragma unroll
            for (int q = 0; q < kRun1; q++) tot = ColT<Real>::add(tot, nxp[q]);
            s_sum[warp][lane] = tot;
            __syncthreads();
            Col run = s_carry[lane];
            for (int w = 0; w < warp; w++) run = ColT<Real>::addc(run, s_sum[w][lane]);
#pragma unroll
            for (int q = 0; q < kRun1; q++) {
                const int m = mb + q;
                if (live && m < R.len) Nout[R.base + (long long)m * R.step] = Real(ColT<Real>::to_real(run) * dx);
                run = ColT<Real>::add(run, nxp[q]);
            }
            __syncthreads();
            if (warp == 7) s_carry[lane] = run;                    // the stretch's end
        } else {
            Col pre[kRun1 + 1];
            pre[0] = ColT<Real>::zero();
#pragma unroll
            for (int q = 0; q < kRun1; q++) {
                const int m = mb + q;
                const bool in = live && m < R.len;
                const long long g = R.base + (long long)(in ? m : 0) * R.step;
                const Real xv = __ldg(x + g), nv = __ldg(nd + g * nmul);
                pre[q + 1] = acc_nx(pre[q], nv, in ? xv : Real(0));
            }
            s_sum[warp][lane] = pre[kRun1];
            __syncthreads();
            Col off = s_carry[lane];
            for (int w = 0; w < warp; w++) off = ColT<Real>::addc(off, s_sum[w][lane]);
            const auto base = col_base(off, dx);
#pragma unroll
            for (int q = 0; q < kRun1; q++) {
                const int m = mb + q;
                if (live && m < R.len) Nout[R.base + (long long)m * R.step] = Real(col_out(base, pre[q], dx));
            }
            __syncthreads();
            if (warp == 7) s_carry[lane] = ColT<Real>::addc(off, pre[kRun1]);
        }
        __syncthreads();
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
    // axis 0: a warp per row; axes 1, 2: 256 threads per 32 rows.  Whole
    // blocks of 256, so that a block never spans two jobs.
    const long long t = (code >> 1) == 0 ? rows * 32 : (rows + 31) / 32 * 256;
    return (t + 255) / 256 * 256;
}

template <typename Real>
cudaError_t launch_plane(const GridDev<Real> *grids, const PlaneJob *jobs, int njobs, int nrow0, long long nthreads,
                         long long threads0, const DevTable<Real> *tabs, int which, int implicit, cudaStream_t s)
{
    if (njobs <= 0 || nthreads <= 0) return cudaSuccess;
    if (implicit) {
        const int bs = 128;
        plane_implicit_kernel<Real><<<(unsigned)((nthreads + bs - 1) / bs), bs, 0, s>>>(grids, jobs, njobs, nthreads,
                                                                                        tabs);
        return cudaGetLastError();
    }
    const int bs = 256;
    if (nrow0 > 0)
        plane_trace_kernel<Real, true><<<(unsigned)((threads0 + bs - 1) / bs), bs, 0, s>>>(grids, jobs, nrow0, 0,
                                                                                          threads0, which);
    if (njobs > nrow0)
        plane_trace_kernel<Real, false><<<(unsigned)((nthreads - threads0 + bs - 1) / bs), bs, 0, s>>>(
            grids, jobs + nrow0, njobs - nrow0, threads0, nthreads, which);
    return cudaGetLastError();
}

template cudaError_t launch_plane<double>(const GridDev<double> *, const PlaneJob *, int, int, long long, long long,
                                          const DevTable<double> *, int, int, cudaStream_t);
template cudaError_t launch_plane<float>(const GridDev<float> *, const PlaneJob *, int, int, long long, long long,
                                         const DevTable<float> *, int, int, cudaStream_t);

} // namespace oots
