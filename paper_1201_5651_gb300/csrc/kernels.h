// Kernel launch interfaces used by the host driver.
#pragma once
#include <cuda_runtime.h>
#include "oots_internal.h"

namespace oots {

template <typename Real> struct DevTable;
struct ff;
template <typename Real> struct ColT;

// Tile shapes of the wavefront sweep: (id, TX, TY, TZ); one chain thread per
// (j,k) column (TY*TZ a multiple of 32) plus one producer warp.  Shapes with
// TY*TZ = 32 keep the whole plane chain in one warp.
#define OOTS_SHAPES(X) \
    X(0, 16, 8, 8)     \
    X(1, 16, 8, 4)     \
    X(2, 16, 16, 16)   \
    X(3, 32, 8, 4)     \
    X(4, 8, 8, 8)      \
    X(5, 16, 16, 8)    \
    X(6, 8, 8, 4)
// Shapes 7 and 8 tile the octants like shapes 4 (8 x 8 x 8) and 0 (16 x 8 x 8)
// but trace them with the throughput kernel (whole tiles, 64 threads, layer
// sweeps off the diagonal planes; sweep_tp.cuh); the implicit sweep (A1) runs
// the pipelined kernel of the same tile (shape 4 or 0) on them.
enum { NUM_SHAPES = 9, SHAPE_TP8 = 7, SHAPE_TP16 = 8 };
static const int SHAPE_DIMS[NUM_SHAPES][3] = {{16, 8, 8}, {16, 8, 4}, {16, 16, 16}, {32, 8, 4}, {8, 8, 8},
                                              {16, 16, 8}, {8, 8, 4}, {8, 8, 8}, {16, 8, 8}};
inline bool is_tp_shape(int shape) { return shape == SHAPE_TP8 || shape == SHAPE_TP16; }
inline int tp_twin(int shape) { return shape == SHAPE_TP8 ? 4 : 0; }   // pipelined kernel on the same tiles

template <typename Real> struct SweepParams {
    const GridDev<Real> *grids;
    const Job *jobs;
    const TileItem *items;
    int nitems;
    int which;                         // 0: trace x into N1; 1: trace xh into N2
    unsigned *ticket;                  // zeroed before each launch
    unsigned *done;                    // CTAs finished; zeroed before each launch
    unsigned *epoch;                   // launches finished so far (persistent; starts at 0)
    unsigned long long *faces;         // per tile 3 faces x FMAX cells x tagged words (zeroed once)
    const DevTable<Real> *tabs;
    int *err;                          // sticky device error
    Real *tpfaces;                     // throughput kernel: per tile 3 faces x tp_face_comps x 64 values
    unsigned *tpflags;                 // throughput kernel: per tile the epoch of the launch that finished it
    long long spin_limit;              // bounded wait on upstream tiles
    long long skip_publish;            // tile that never writes its faces (fault-injection test), -1: none
    int chunk;                         // planes per hand-off chunk (<= 0: 4)
    int ngrid;                         // grids in `grids` (> 0: the launch returns at once when every
                                       // grid has reached its end time; 0: no such check)
    const void *bricks;                // throughput kernel: base of the packed n x of every grid, brick
                                       // TileItem::brick at bricks + brick x TX x 64 values (nullptr: none)
};

// tagged 8-byte words per published face cell (mixed path 3, FP64 path 4)
template <typename Real> constexpr int face_words() { return sizeof(Real) == 4 ? 3 : 4; }
// values per face cell the throughput kernel publishes: the column (float-float
// hi and lo in the mixed path, one double in FP64) and the weight factor
template <typename Real> __host__ __device__ constexpr int tp_face_comps() { return sizeof(Real) == 4 ? 3 : 2; }

template <typename Real> cudaError_t prepare_sweeps();
template <typename Real> int sweep_occupancy(int shape, int mode);   // resident CTAs per SM
template <typename Real> bool sweep_shape_ok(int shape);              // fits the shared memory of this device
template <typename Real>
cudaError_t launch_sweep(const SweepParams<Real> &P, int shape, int mode, int nblocks, cudaStream_t s);
// n x of the traced state (which = 0: x, 1: xh) into each grid's bricks (GridDev::nxb) for the
// throughput kernel of tile shape `shape`; max_elems = the largest grid's brick cells
template <typename Real>
cudaError_t launch_pack_nx(const GridDev<Real> *grids, int ngrid, int which, int shape, long long max_elems, int nsm,
                           cudaStream_t s);

// Plane-parallel sources: which = 0 traces x into N1, 1 traces xh into N2;
// implicit = 1 runs the A1 row integration instead (single source).  The jobs
// along x come first (nrow0 of them, threads0 threads); nthreads is the sum
// of plane_job_threads over all jobs, whose `first` fields are the running
// sums.
long long plane_job_threads(int code, long long rows);
template <typename Real>
cudaError_t launch_plane(const GridDev<Real> *grids, const PlaneJob *jobs, int njobs, int nrow0, long long nthreads,
                         long long threads0, const DevTable<Real> *tabs, int which, int implicit, cudaStream_t s);

// Per-cell passes.  HALF and FULL run as a closed-form pass over all cells
// followed by the general pass (op | OP_GENERAL) over the queued cells.
enum { OP_RATEDT = 0, OP_HALF = 1, OP_FULL1 = 2, OP_FULL2 = 3, OP_RATEDT_VERIFY = 4, OP_GENERAL = 16 };
// qrec: per queue slot the closed-form pass's rates and f(x0) of single-source
// cells (queue_record_bytes each), so the general pass starts at the root
// search (unused, may be null, when nsmax > 1).  rcache: 3 x total values per
// cell that the dt pass writes and the half step (A3) or full step (A2) of
// the same substep reads when use_cache is set: the transmitted fraction,
// F(x0) and F'(x0) of single-source grids; F(x0), F'(x0) and the sum of the
// sources' rate bounds when nsmax > 1 (the full step then recomputes).
// cell_bs: threads per block of the closed-form passes, 128 or 256 (the general passes use 256).
template <typename Real>
cudaError_t launch_cell(const GridDev<Real> *grids, int ngrid, const long long *offsets, long long total,
                        const DevTable<Real> *tabs, int op, int nsmax, unsigned *queue, unsigned *qcount,
                        Real *qrec, Real *rcache, int use_cache, int gen_blocks, int cell_bs, cudaStream_t s);
template <typename Real> size_t queue_record_bytes();
template <typename Real> int cell_general_occupancy(int nsmax);
// stage 0 also clears the queue lengths and the general passes' head counters
template <typename Real>
cudaError_t launch_finalize(const GridDev<Real> *grids, int ngrid, int stage, unsigned *qcount,
                            const DevTable<Real> *tabs, cudaStream_t s);

} // namespace oots
