// Internal types shared by the host driver and the CUDA kernels.
#pragma once
#include <stdint.h>

namespace oots {

enum { MAX_SRC = 64 };          // sources per grid

// Device-side error codes written to DevState::err (first one sticks).
enum { DEVERR_NONE = 0, DEVERR_TIMEOUT = 1, DEVERR_BOUNDS = 2 };

// One (grid, source, octant) sweep: the octant of cells on one side of the
// source vertex along each axis, traced outward from the vertex (Sect. 5).
struct Job {
    int grid;              // index into the launch's grid array
    int src;               // source index within the grid
    int v[3];              // source vertex
    int sg[3];             // octant signs (+1 / -1)
    int ext[3];            // octant extent in cells
    int off[3];            // tile offset: octant-local i of tile I starts at I*T - off
    int nt[3];             // tiles per axis
    long long tile_base;   // index of tile (0,0,0) in the flag and face arrays
};

// One plane-parallel source of one grid (a source at infinity whose rays run
// along a grid axis, Sect. 3.1): its rows are traced independently (the
// thread layout per axis is in plane.cu).
struct PlaneJob {
    int grid;              // index into the launch's grid array
    int src;               // source index within the grid
    int code;              // 2*axis + back: rays along +axis (back 0) or -axis (back 1)
    int pad;
    long long rows;        // rows of cells parallel to the axis
    long long first;       // first thread of the job in the launch (a multiple of 256)
};

// One tile of a job, ordered in the work list by tile diagonal I+J+K.  grid:
// the job's grid (as Job::grid; launches of at most 65535 grids).  brick: the
// tile's brick in the launch's packed n x (GridDev::nxb counts from the same
// base), when the launch packs its input (throughput tiles).
struct TileItem { int job; unsigned short I, J, K, grid; unsigned brick; };

// Per-grid state that lives on the device, read and written by the kernels
// (so that substeps can be replayed from a CUDA graph without host sync).
struct DevState {
    double t, t_end;          // current time, end of the advance
    double dt;                // timestep of the substep in flight (0: done)
    double dt_last;           // the last nonzero timestep (the dt pass's hint)
    double dt_fixed;          // > 0: fixed timestep
    double K1, K3, K4;        // Eq. 4 factors (<= 0: off)
    unsigned long long dt_bits;   // min over cells of the criterion (bits of a positive double)
    double sumQ;              // sum of the source rates [1/s]
    double bud_step[4];       // emitted, absorbed, new ions, recombinations of the last substep
    double bud_total[4];      // accumulated since the last reset
    double cell_volume;       // dx^3
    long long nsub;           // substeps taken
    int done;                 // t >= t_end
    int err;                  // DEVERR_*
    float lnthr[4];           // source-selection thresholds ln(1e-3 eps / H), set with each step: the next
                              // dt pass's (H = 4 dt_last; used while dt_last > 0), the half step's
                              // (H = dt/2) and the full step's (H = dt); [3] unused
};

// What the many-source passes read of one source to decide whether it can
// matter at a cell (Mackey 2012 Sect. 2 rate, bounded): one record of a few
// 16-byte words instead of a dozen scattered descriptor reads.
template <typename Real> struct __align__(16) SrcSel {
    Real nst;                // negligible column of the pass (+inf: none)
    Real N0, Nhi;            // tabulated: first and last node column
    const Real *L;           // tabulated: node values ln(P/Q)
    float lnamp0;            // ln(qfac sigma0 dx)
    float lnN_lo, inv_dl;    // tabulated: table axis (as float)
    float msig;              // monochromatic: -sigma0 (as float)
    int v0, v1, v2;          // vertex
    int K;                   // tabulated: nodes; -1: monochromatic
    int plane;               // plane-parallel source
};

// Description of one grid for the kernels (Real = float or double).
template <typename Real> struct GridDev {
    int nx, ny, nz;
    long long ncell;
    long long cell_lo, cell_hi;   // the per-cell passes update cells [cell_lo, cell_hi) of the grid
    Real dx;
    Real sigma0, tau0, alpha;
    const Real *n;            // density (nullptr: uniform n_uniform)
    Real n_uniform;
    const Real *x;            // state the sweep traces / the cell kernels start from
    const Real *xh;           // half-step state (A3 second sweep input)
    Real *xout;               // where the cell kernels write
    Real *N1;                 // entry columns of the first trace, nsrc x ncell
    Real *N2;                 // entry columns of the second trace, nsrc x ncell
    int nsrc;
    int vtx[MAX_SRC][3];
    Real qfac[MAX_SRC];       // Q / (4 pi dx^3); a plane source's flux F / dx
    int tab[MAX_SRC];         // -1 monochromatic, else table index
    unsigned char pcode[MAX_SRC];  // 0: vertex point source; 1 + 2*axis + back: plane source (qfac = F/dx)
    float lnamp0[MAX_SRC];    // ln(qfac sigma0 dx): a source's largest rate per unit x is qfac sigma0 dx p / r2
    Real *nxb;                // n x of the traced state in bricks of the throughput tile (nullptr: none):
                              // brick (bx, by, bz) of nbx x nby x nbz holds cells bx*TX.., by*8.., bz*8..,
                              // x fastest, TX = the tile's x extent
    int nbx, nby, nbz;
    SrcSel<Real> *sel;        // 4 x MAX_SRC source records for the dt pass (nst: the column beyond which
                              // a source cannot matter within the step hint), the half step, the full
                              // step and the verifying dt pass (nst = +inf); nullptr: one source
    DevState *st;
};

} // namespace oots
