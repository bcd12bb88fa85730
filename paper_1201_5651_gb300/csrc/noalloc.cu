// oots_trace_noalloc: the column-density trace for callers that cannot
// allocate device memory.  It runs the same wavefront sweep kernel as the
// context API, but every piece of scratch it needs (the tile work list, the
// published tile faces and the small descriptors) lives in
// one file-scope static device array, so the call makes no cudaMalloc, no
// cudaFree and no heap allocation on the host.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/oots.h"
#include "common.cuh"
#include "kernels.h"

using namespace oots;

// error text for oots_last_error (defined with the rest of the C ABI)
void oots_set_error_text(const char *msg);

namespace {

// 64 MiB, resident on every device that loads the library until the process exits.
constexpr size_t kScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kShape = 0;                       // tile shape 16 x 8 x 8
constexpr int kTX = 16, kTY = 8, kTZ = 8;
constexpr int kFMAX = 128;                      // largest face of the tile
constexpr int kMaxDiag = 4096;                  // tile diagonals the work-list builder can order
constexpr size_t kHeader = 64 * 1024;           // ticket, error, state, counters

// header layout (byte offsets inside the scratch)
constexpr size_t kOffTicket = 0;                // ticket, then the count of finished CTAs
constexpr size_t kOffEpoch = 64;                // sweep launches so far: never cleared (faces carry it)
constexpr size_t kOffErr = 128;
constexpr size_t kOffState = 256;               // DevState (done = 0 after the clear)
constexpr size_t kOffCount = 1024;              // kMaxDiag unsigned: tiles per diagonal, then cursor
constexpr size_t kOffJobs = kOffCount + 2 * kMaxDiag * sizeof(unsigned);
constexpr size_t kOffGrid = kOffJobs + 8 * sizeof(Job) + 256;

struct DevSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;
    int nblocks[2] = {0, 0};   // per precision
};
static DevSetup g_setup[64];
static std::mutex g_setup_mutex;   // first-call set-up of a device, from any host thread

template <typename Real> size_t tile_bytes()
{
    return sizeof(TileItem) + 3 * kFMAX * face_words<Real>() * sizeof(unsigned long long);
}

// Byte offset of the per-tile arrays, and the most tiles the scratch holds
// after them (one item slot is kept spare).
template <typename Real> size_t tiles_offset()
{
    return (kOffGrid + sizeof(GridDev<Real>) + 255) / 256 * 256;
}
template <typename Real> long long max_tiles()
{
    return (long long)((kScratchBytes - tiles_offset<Real>()) / tile_bytes<Real>()) - 1;
}

// One block orders the tiles of the (at most 8) octant jobs by tile diagonal:
// count per diagonal, exclusive scan, then place (order inside a diagonal is free).
__global__ void build_worklist(const Job *jobs, int njobs, unsigned *count, unsigned *cursor, TileItem *items,
                               int maxdiag)
{
    for (int d = threadIdx.x; d < maxdiag; d += blockDim.x) { count[d] = 0u; cursor[d] = 0u; }
    __syncthreads();
    for (int j = 0; j < njobs; j++) {
        const Job J = jobs[j];
        const long long n = (long long)J.nt[0] * J.nt[1] * J.nt[2];
        for (long long t = threadIdx.x; t < n; t += blockDim.x) {
            const int I = (int)(t % J.nt[0]), Jj = (int)((t / J.nt[0]) % J.nt[1]), K = (int)(t / ((long long)J.nt[0] * J.nt[1]));
            atomicAdd(&count[I + Jj + K], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int d = 0; d < maxdiag; d++) { const unsigned c = count[d]; cursor[d] = acc; acc += c; }
    }
    __syncthreads();
    for (int j = 0; j < njobs; j++) {
        const Job J = jobs[j];
        const long long n = (long long)J.nt[0] * J.nt[1] * J.nt[2];
        for (long long t = threadIdx.x; t < n; t += blockDim.x) {
            const int I = (int)(t % J.nt[0]), Jj = (int)((t / J.nt[0]) % J.nt[1]), K = (int)(t / ((long long)J.nt[0] * J.nt[1]));
            const unsigned pos = atomicAdd(&cursor[I + Jj + K], 1u);
            TileItem it;
            it.job = j;
            it.I = (unsigned short)I;
            it.J = (unsigned short)Jj;
            it.K = (unsigned short)K;
            it.grid = 0;
            it.brick = 0u;
            items[pos] = it;
        }
    }
}

template <typename Real>
int trace_noalloc(DevSetup &S, int nx, int ny, int nz, double dx, const void *n_dev, double n_uniform,
                  const void *x_dev, const int vtx[3], double sigma0, double tau0, void *Nin_dev, cudaStream_t st)
{
    const int n3[3] = {nx, ny, nz};
    const int T3[3] = {kTX, kTY, kTZ};
    Job jobs[8];
    int njobs = 0;
    long long tiles = 0;
    int maxd = 0;
    for (int o = 0; o < 8; o++) {
        Job J;
        memset(&J, 0, sizeof(J));
        J.grid = 0;
        J.src = 0;
        bool empty = false;
        for (int a = 0; a < 3; a++) {
            J.v[a] = vtx[a];
            J.sg[a] = (o >> a) & 1 ? -1 : 1;
            J.ext[a] = J.sg[a] > 0 ? n3[a] - vtx[a] : vtx[a];
            if (J.ext[a] <= 0) empty = true;
            const int r = vtx[a] % T3[a];
            J.off[a] = J.sg[a] > 0 ? r : (T3[a] - r) % T3[a];
            J.nt[a] = (J.ext[a] + J.off[a] + T3[a] - 1) / T3[a];
        }
        if (empty) continue;
        J.tile_base = tiles;
        tiles += (long long)J.nt[0] * J.nt[1] * J.nt[2];
        const int d = J.nt[0] + J.nt[1] + J.nt[2] - 2;
        if (d > maxd) maxd = d;
        jobs[njobs++] = J;
    }
    const long long maxt = max_tiles<Real>();
    if (tiles > maxt || maxd + 1 > kMaxDiag)
        return -1000 - (int)std::min<long long>(tiles, 1 << 30);   // reported by the caller

    unsigned char *sc = S.scratch;
    // layout of the per-tile arrays after the fixed part
    size_t off = tiles_offset<Real>();
    TileItem *items = (TileItem *)(sc + off);
    off += (size_t)(maxt + 1) * sizeof(TileItem);
    off = (off + 255) / 256 * 256;
    unsigned long long *faces = (unsigned long long *)(sc + off);   // zero at load; launches tag epochs 1, 2, ...

    GridDev<Real> G;
    memset(&G, 0, sizeof(G));
    G.nx = nx; G.ny = ny; G.nz = nz;
    G.ncell = (long long)nx * ny * nz;
    G.cell_lo = 0;
    G.cell_hi = G.ncell;
    G.dx = Real(dx);
    G.sigma0 = Real(sigma0);
    G.tau0 = Real(tau0);
    G.n = (const Real *)n_dev;
    G.n_uniform = Real(n_uniform);
    G.x = (const Real *)x_dev;
    G.xh = (const Real *)x_dev;
    G.N1 = (Real *)Nin_dev;
    G.nsrc = 1;
    for (int a = 0; a < 3; a++) G.vtx[0][a] = vtx[a];
    G.tab[0] = -1;
    G.st = (DevState *)(sc + kOffState);

    // clear what must start at zero: ticket, finished-CTA count, error, device state
    // (the epoch and the faces are never cleared: stale face words carry older epochs)
    if (cudaMemsetAsync(sc + kOffTicket, 0, kOffEpoch - kOffTicket, st) != cudaSuccess) return -1;
    if (cudaMemsetAsync(sc + kOffErr, 0, kOffCount - kOffErr, st) != cudaSuccess) return -1;
    if (cudaMemcpyAsync(sc + kOffJobs, jobs, njobs * sizeof(Job), cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
    if (cudaMemcpyAsync(sc + kOffGrid, &G, sizeof(G), cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
    if (tiles == 0) return 0;
    build_worklist<<<1, 1024, 0, st>>>((const Job *)(sc + kOffJobs), njobs, (unsigned *)(sc + kOffCount),
                                       (unsigned *)(sc + kOffCount) + kMaxDiag, items, maxd + 1);
    if (cudaGetLastError() != cudaSuccess) return -1;

    SweepParams<Real> P;
    P.grids = (const GridDev<Real> *)(sc + kOffGrid);
    P.jobs = (const Job *)(sc + kOffJobs);
    P.items = items;
    P.nitems = (int)tiles;
    P.which = 0;
    P.ticket = (unsigned *)(sc + kOffTicket);
    P.done = (unsigned *)(sc + kOffTicket) + 1;
    P.epoch = (unsigned *)(sc + kOffEpoch);
    P.faces = faces;
    P.tpfaces = nullptr;
    P.tpflags = nullptr;
    P.tabs = nullptr;
    P.err = (int *)(sc + kOffErr);
    P.spin_limit = 1ll << 22;
    P.skip_publish = -1;
    P.chunk = 0;
    P.ngrid = 0;
    P.bricks = nullptr;
    const int prec = sizeof(Real) == 8 ? 0 : 1;
    if (launch_sweep<Real>(P, kShape, 0, S.nblocks[prec], st) != cudaSuccess) return -1;
    return 0;
}

} // namespace

extern "C" int oots_trace_noalloc(int device, int precision, int nx, int ny, int nz, double dx_cm,
                                  const void *n_dev, double uniform_n, const void *x_dev, const double pos_cells[3],
                                  double sigma0, double tau0, void *Nin_dev, void *stream, int *status_detail)
{
    if (status_detail) *status_detail = 0;
    if (precision != OOTS_FP64 && precision != OOTS_MIXED) return OOTS_E_INVAL;
    if (nx <= 0 || ny <= 0 || nz <= 0 || nx > 8192 || ny > 8192 || nz > 8192) return OOTS_E_INVAL;
    if (!(dx_cm > 0) || !std::isfinite(dx_cm) || !(sigma0 > 0) || !(tau0 > 0)) return OOTS_E_INVAL;
    if (!x_dev || !Nin_dev || !pos_cells) return OOTS_E_INVAL;
    if (!n_dev && !(uniform_n > 0)) return OOTS_E_INVAL;
    if (device < 0 || device >= 64) return OOTS_E_INVAL;
    int vtx[3];
    const int n3[3] = {nx, ny, nz};
    for (int a = 0; a < 3; a++) {
        if (!std::isfinite(pos_cells[a])) return OOTS_E_INVAL;
        double v = std::floor(pos_cells[a] + 0.5);
        vtx[a] = (int)std::min<double>(std::max<double>(v, 0.0), n3[a]);
    }
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return OOTS_E_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return OOTS_E_CUDA;
    DevSetup &S = g_setup[device];
    int rc = OOTS_OK;
    std::unique_lock<std::mutex> setup_lock(g_setup_mutex);
    if (!S.ready) {
        // once per device, with the device current: the device address of the
        // static scratch (its host-side name is only a stand-in), the kernels'
        // shared-memory opt-in, and the persistent grid size
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) rc = OOTS_E_CUDA;
        if (rc == OOTS_OK && (prepare_sweeps<double>() != cudaSuccess || prepare_sweeps<float>() != cudaSuccess))
            rc = OOTS_E_CUDA;
        if (rc == OOTS_OK) {
            int nsm = 0;
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
            S.scratch = (unsigned char *)p;
            S.nblocks[0] = sweep_occupancy<double>(kShape, 0) * nsm;
            S.nblocks[1] = sweep_occupancy<float>(kShape, 0) * nsm;
            S.ready = true;
        }
    }
    setup_lock.unlock();
    cudaStream_t st = (cudaStream_t)stream;
    if (rc == OOTS_OK) {
        int r = precision == OOTS_FP64
                    ? trace_noalloc<double>(S, nx, ny, nz, dx_cm, n_dev, uniform_n, x_dev, vtx, sigma0, tau0, Nin_dev, st)
                    : trace_noalloc<float>(S, nx, ny, nz, dx_cm, n_dev, uniform_n, x_dev, vtx, sigma0, tau0, Nin_dev, st);
        if (r <= -1000) {
            if (status_detail) *status_detail = -1000 - r;   // tiles the problem needs
            char msg[256];
            snprintf(msg, sizeof(msg),
                     "oots_trace_noalloc: the grid needs %d tiles of 16x8x8 cells; the %zu MiB static scratch holds "
                     "at most %lld (%s)", -1000 - r, kScratchBytes >> 20,
                     precision == OOTS_FP64 ? max_tiles<double>() : max_tiles<float>(),
                     precision == OOTS_FP64 ? "FP64" : "mixed");
            oots_set_error_text(msg);
            rc = OOTS_E_INVAL;
        } else if (r != 0) {
            rc = OOTS_E_CUDA;
        } else {
            int err = 0;
            if (cudaMemcpyAsync(&err, S.scratch + kOffErr, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = OOTS_E_CUDA;
            else if (err == DEVERR_TIMEOUT)
                rc = OOTS_E_DEVICE_TIMEOUT;
        }
    }
    cudaSetDevice(prev);
    return rc;
}
