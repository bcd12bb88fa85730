// C ABI of the library (include/oots.h): argument checking, device memory,
// source snapping and octant split, the tile work list, substep sequencing
// of the schemes A1/A2/A3 (Mackey 2012, Sect. 2.1-2.2) and CUDA-graph replay.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/oots.h"
#include "common.cuh"
#include "kernels.h"
#include "tables.h"

using namespace oots;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err = "no error";

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void oots_set_error_text(const char *msg) { g_err = msg; }

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(OOTS_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct SourceH {
    double pos[3];
    int v[3];
    double Q;              // photons per second; a plane source's flux per unit area
    int spectrum;
    double T;
    int pcode = 0;         // 0: vertex point source; 1 + 2*axis + back: plane source
};

// Photons per second a source sends into the grid: a plane source's flux
// times the area of the face it enters through.
static double source_emission(const SourceH &S, int nx, int ny, int nz, double dx)
{
    if (!S.pcode) return S.Q;
    const int n3[3] = {nx, ny, nz};
    const int axis = (S.pcode - 1) >> 1;
    return S.Q * (double)n3[(axis + 1) % 3] * (double)n3[(axis + 2) % 3] * dx * dx;
}

// Optional per-launch timing (oots_profile_substep): events around each launch.
struct LaunchProfiler {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kinds;
    cudaStream_t s = nullptr;
    void mark(int kind)
    {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev.push_back(e);
        kinds.push_back(kind);
    }
    ~LaunchProfiler()
    {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

struct LaunchSetBase {
    LaunchProfiler *prof = nullptr;
    virtual ~LaunchSetBase() {}
    virtual int substep(cudaStream_t s, bool fixed_dt) = 0;
    virtual int trace_for_dt(cudaStream_t s) = 0;
    virtual int graph_replay(cudaStream_t s, int n) = 0;
    // one phase of a substep, eagerly (partitioned runs): 0 trace x, 1 dt pass,
    // 2 choose dt and half step (A3; A2: full step), 3 trace x_half, 4 full step (A3)
    virtual int phase(cudaStream_t s, int ph, bool use_cache) = 0;
};

struct oots_ctx {
    int device = 0, precision = OOTS_FP64;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    int nx = 0, ny = 0, nz = 0;
    double dx = 0.0;
    long long ncell = 0;
    double alpha = 2.59e-13, sigma0 = 6.3e-18, tau0 = 0.6, T = 1e4;
    bool uniform_n = true;
    double n_uniform = 1.0;
    std::vector<SourceH> src;
    int scheme = OOTS_A3;
    oots_dtcrit crit = {0.0, 0.0, 0.0, 0.25, 0.0};
    int shape = -1;
    long long spin_limit = 1ll << 22;
    long long skip_publish = -1;
    int sweep_chunk = 0;               // planes per progress step of the sweep (0: default)
    int tile_align = 0;                // tile origins: 0 global multiples of the tile (x rows aligned), 1 the octant's
    int cell_block = 0;                // threads per block of the closed-form passes: 128, 256, 0 = by source count
    size_t rsize = 8;
    void *d_x = nullptr, *d_n = nullptr, *d_xh = nullptr, *d_N1 = nullptr, *d_N2 = nullptr;
    void *d_stage = nullptr;           // ncell doubles: host arrays pass through it (allocated on first use)
    long long *d_bad = nullptr;        // first cell a device-side check rejected
    int nsrc_alloc = 0;
    DevState *d_st = nullptr;
    int *d_err = nullptr;
    DevState h_st;
    unsigned long long part_src = ~0ull;   // partition: sources this context traces (bit s)
    int part_z0 = 0, part_z1 = 0;          // partition: z-range of the cells it updates (z1 <= 0: all)
    bool phase_dt = false;                 // the dt phase ran on the current columns
    LaunchSetBase *solo = nullptr;
    bool dirty = true;      // sources / grid / shape / scheme changed since the launch set was built
    int nsm = 0;
    bool batched = false;
};

static size_t rsz(int precision) { return precision == OOTS_FP64 ? sizeof(double) : sizeof(float); }

static void free_dev(void *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// ---------------------------------------------------------------------------
// Launch set: everything one substep of a group of contexts needs on the device
// ---------------------------------------------------------------------------
template <typename Real> struct LaunchSet : LaunchSetBase {
    std::vector<oots_ctx *> ctxs;
    int device = 0;
    int shape = 0;
    int scheme = OOTS_A3;
    GridDev<Real> *d_grids = nullptr;
    Job *d_jobs = nullptr;
    TileItem *d_items = nullptr;
    int nitems = 0;
    long long ntiles = 0;
    unsigned *d_sync = nullptr;        // [0] ticket, [1] done (zeroed per sweep), [16] epoch (persistent)
    unsigned long long *d_faces = nullptr;
    Real *d_tpfaces = nullptr;         // throughput sweep: untagged faces, and a flag per tile
    unsigned *d_tpflags = nullptr;
    Real *d_bricks = nullptr;          // throughput sweep: n x of every grid in bricks of the tile
    long long brick_max = 0;           // brick cells of the largest grid (0: no bricks)
    PlaneJob *d_pjobs = nullptr;       // plane-parallel sources
    int npjobs = 0, nrow0 = 0;         // jobs; of them, rows along x (first in the array)
    long long plane_threads = 0, threads0 = 0;
    DevTable<Real> *d_tabs = nullptr;
    std::vector<void *> tabmem;
    long long *d_offsets = nullptr;
    long long total = 0;
    unsigned *d_queue = nullptr;       // cells left to the general pass (one entry per cell at most)
    Real *d_qrec = nullptr;            // their closed-form results (single-source launch sets)
    Real *d_rcache = nullptr;          // per cell: transmitted fraction, F(x0), F'(x0) from the dt pass
    SrcSel<Real> *d_sel = nullptr;     // per grid 4 x MAX_SRC source records of the selection (several sources)
    unsigned *d_qcount = nullptr;      // queue lengths of the half and full integrations
    int gen_blocks = 1;                // grid of the general pass
    int cell_bs = 128;                 // threads per block of the closed-form passes
    int nblocks0 = 1, nblocks1 = 1;
    int nsmax = 1;                     // largest source count among the grids
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_fixed = false;
    int *d_err = nullptr;
    long long spin_limit = 1ll << 22, skip_publish = -1;
    int sweep_chunk = 0;

    ~LaunchSet() override
    {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(d_grids);
        cudaFree(d_jobs);
        cudaFree(d_items);
        cudaFree(d_sync);
        cudaFree(d_faces);
        cudaFree(d_tpfaces);
        cudaFree(d_tpflags);
        cudaFree(d_pjobs);
        cudaFree(d_tabs);
        for (void *p : tabmem) cudaFree(p);
        cudaFree(d_bricks);
        cudaFree(d_offsets);
        cudaFree(d_queue);
        cudaFree(d_qrec);
        cudaFree(d_rcache);
        cudaFree(d_sel);
        cudaFree(d_qcount);
    }

    int upload_table(const HostTable &H, DevTable<Real> &T)
    {
        std::vector<Real> coef(H.coef.begin(), H.coef.end()), L(H.L.begin(), H.L.end()),
            Nn(H.Nnode.begin(), H.Nnode.end());
        Real *dc = nullptr, *dL = nullptr, *dN = nullptr;
        CU(cudaMalloc(&dc, coef.size() * sizeof(Real)));
        tabmem.push_back(dc);
        CU(cudaMalloc(&dL, L.size() * sizeof(Real)));
        tabmem.push_back(dL);
        CU(cudaMalloc(&dN, Nn.size() * sizeof(Real)));
        tabmem.push_back(dN);
        CU(cudaMemcpy(dc, coef.data(), coef.size() * sizeof(Real), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(dL, L.data(), L.size() * sizeof(Real), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(dN, Nn.data(), Nn.size() * sizeof(Real), cudaMemcpyHostToDevice));
        T.coef = dc;
        T.L = dL;
        T.Nnode = dN;
        T.lnN_lo = Real(H.lnN_lo);
        T.dl = Real(H.dl);
        T.inv_dl = Real(1.0 / H.dl);
        T.N0 = Real(H.Nnode[0]);
        T.Nhi = Real(H.Nnode[H.K - 1]);
        T.a0 = Real(H.a0);
        T.K = H.K;
        return OOTS_OK;
    }

    int build(const std::vector<oots_ctx *> &cs, int shape_req)
    {
        ctxs = cs;
        if (cs.size() > 65535) return fail(OOTS_E_INVAL, "%zu grids in one call (at most 65535)", cs.size());
        oots_ctx *c0 = cs[0];
        device = c0->device;
        scheme = c0->scheme;
        shape = shape_req >= 0 ? shape_req : 0;
        if (!sweep_shape_ok<Real>(shape))
            return fail(OOTS_E_UNSUPPORTED, "tile shape %d does not fit in shared memory at this precision", shape);
        d_err = c0->d_err;
        spin_limit = c0->spin_limit;
        skip_publish = c0->skip_publish;
        sweep_chunk = c0->sweep_chunk;
        const int TX = SHAPE_DIMS[shape][0], TY = SHAPE_DIMS[shape][1], TZ = SHAPE_DIMS[shape][2];
        const int T3[3] = {TX, TY, TZ};
        const int FMAX = std::max(TY * TZ, std::max(TX * TZ, TX * TY));

        std::vector<GridDev<Real>> grids(cs.size());
        std::vector<Job> jobs;
        std::vector<PlaneJob> pjobs;
        std::vector<TileItem> items;
        std::vector<DevTable<Real>> tabs;
        std::vector<long long> offs(cs.size());
        long long tile_base = 0, off = 0;
        // the throughput kernel's traces read n x packed in bricks of the tile
        // (tiles at global multiples of the tile only), one allocation for all grids
        const bool pack = is_tp_shape(shape) && scheme != OOTS_A1;
        std::vector<long long> brick_base(cs.size(), -1);
        long long nbricks = 0;
        for (size_t g = 0; g < cs.size(); g++) {
            oots_ctx *c = cs[g];
            GridDev<Real> &G = grids[g];
            memset(&G, 0, sizeof(G));
            if (pack && !c->tile_align) {
                G.nbx = (c->nx + TX - 1) / TX;
                G.nby = (c->ny + TY - 1) / TY;
                G.nbz = (c->nz + TZ - 1) / TZ;
                brick_base[g] = nbricks;
                nbricks += (long long)G.nbx * G.nby * G.nbz;
            }
            G.nx = c->nx; G.ny = c->ny; G.nz = c->nz;
            G.ncell = c->ncell;
            {
                const long long plane = (long long)c->nx * c->ny;
                const int z1 = c->part_z1 > 0 ? std::min(c->part_z1, c->nz) : c->nz;
                G.cell_lo = plane * std::max(c->part_z0, 0);
                G.cell_hi = plane * z1;
            }
            G.dx = Real(c->dx);
            G.sigma0 = Real(c->sigma0);
            G.tau0 = Real(c->tau0);
            G.alpha = Real(c->alpha);
            G.n = c->uniform_n ? nullptr : (const Real *)c->d_n;
            G.n_uniform = Real(c->n_uniform);
            G.x = (const Real *)c->d_x;
            G.xh = (const Real *)c->d_xh;
            G.xout = (Real *)c->d_x;
            G.N1 = (Real *)c->d_N1;
            G.N2 = (Real *)c->d_N2;
            G.nsrc = (int)c->src.size();
            if (G.nsrc > nsmax) nsmax = G.nsrc;
            G.st = c->d_st;
            for (int s = 0; s < G.nsrc; s++) {
                const SourceH &S = c->src[s];
                for (int a = 0; a < 3; a++) G.vtx[s][a] = S.pcode ? 0 : S.v[a];
                const double qf = S.pcode ? S.Q / c->dx : S.Q / (4.0 * M_PI * c->dx * c->dx * c->dx);
                G.qfac[s] = Real(qf);
                G.lnamp0[s] = (float)std::log(qf * c->sigma0 * c->dx);
                G.pcode[s] = (unsigned char)S.pcode;
                if (S.spectrum == OOTS_MONO) G.tab[s] = -1;
                else {
                    DevTable<Real> T;
                    int rc = upload_table(host_table(1, S.T, c->sigma0), T);
                    if (rc) return rc;
                    G.tab[s] = (int)tabs.size();
                    tabs.push_back(T);
                }
                const int n3[3] = {c->nx, c->ny, c->nz};
                if (s < 64 && !((c->part_src >> s) & 1ull)) continue;   // traced by another process
                if (S.pcode) {
                    PlaneJob P;
                    memset(&P, 0, sizeof(P));
                    P.grid = (int)g;
                    P.src = s;
                    P.code = S.pcode - 1;
                    const int axis = P.code >> 1;
                    P.rows = (long long)n3[(axis + 1) % 3] * n3[(axis + 2) % 3];
                    pjobs.push_back(P);
                    continue;
                }
                for (int o = 0; o < 8; o++) {
                    Job J;
                    memset(&J, 0, sizeof(J));
                    J.grid = (int)g;
                    J.src = s;
                    bool empty = false;
                    for (int a = 0; a < 3; a++) {
                        J.v[a] = S.v[a];
                        J.sg[a] = (o >> a) & 1 ? -1 : 1;
                        J.ext[a] = J.sg[a] > 0 ? n3[a] - S.v[a] : S.v[a];
                        if (J.ext[a] <= 0) empty = true;
                        const int r = S.v[a] % T3[a];
                        J.off[a] = c->tile_align ? 0 : (J.sg[a] > 0 ? r : (T3[a] - r) % T3[a]);
                        J.nt[a] = (J.ext[a] + J.off[a] + T3[a] - 1) / T3[a];
                    }
                    if (empty) continue;
                    J.tile_base = tile_base;
                    const int jid = (int)jobs.size();
                    for (int K = 0; K < J.nt[2]; K++)
                        for (int Jj = 0; Jj < J.nt[1]; Jj++)
                            for (int I = 0; I < J.nt[0]; I++) {
                                TileItem t;
                                t.job = jid;
                                t.I = (unsigned short)I;
                                t.J = (unsigned short)Jj;
                                t.K = (unsigned short)K;
                                t.grid = (unsigned short)g;
                                t.brick = 0u;
                                if (brick_base[g] >= 0) {
                                    // lowest global cell of the tile along each axis (a multiple of the tile)
                                    const int idx3[3] = {I, Jj, K};
                                    long long b3[3];
                                    for (int a = 0; a < 3; a++) {
                                        const int o0 = idx3[a] * T3[a] - J.off[a];
                                        const int lo = J.sg[a] > 0 ? J.v[a] + o0 : J.v[a] - o0 - T3[a];
                                        b3[a] = lo / T3[a];
                                    }
                                    t.brick = (unsigned)(brick_base[g] + (b3[2] * G.nby + b3[1]) * G.nbx + b3[0]);
                                }
                                items.push_back(t);
                            }
                    tile_base += (long long)J.nt[0] * J.nt[1] * J.nt[2];
                    jobs.push_back(J);
                }
            }
            offs[g] = off;
            off += c->ncell;
        }
        total = off;
        ntiles = tile_base;
        nitems = (int)items.size();
        std::stable_sort(items.begin(), items.end(), [](const TileItem &a, const TileItem &b) {
            return a.I + a.J + a.K < b.I + b.J + b.K;
        });

        CU(cudaSetDevice(device));
        if (nbricks > 0 && !jobs.empty()) {
            if (nbricks > 0xffffffffll) return fail(OOTS_E_INVAL, "%lld bricks in one call (32-bit brick indices)", nbricks);
            const long long bc = (long long)TX * TY * TZ;
            CU(cudaMalloc(&d_bricks, (size_t)(nbricks * bc) * sizeof(Real)));
            for (size_t g = 0; g < cs.size(); g++) {
                if (brick_base[g] < 0) continue;
                GridDev<Real> &G = grids[g];
                G.nxb = d_bricks + brick_base[g] * bc;
                brick_max = std::max(brick_max, (long long)G.nbx * G.nby * G.nbz * bc);
            }
        } else {
            for (auto &G : grids) G.nbx = G.nby = G.nbz = 0;
        }
        if (nsmax > 1) {
            // each source's selection record, four copies per grid (dt pass, half step, full
            // step, verifying dt pass); no negligible column until the first step sets them
            const size_t nn = grids.size() * 4 * MAX_SRC;
            std::vector<SrcSel<Real>> sel(nn);
            memset(sel.data(), 0, nn * sizeof(SrcSel<Real>));
            for (size_t g = 0; g < grids.size(); g++) {
                const GridDev<Real> &G = grids[g];
                for (int s = 0; s < G.nsrc; s++) {
                    SrcSel<Real> S;
                    memset(&S, 0, sizeof(S));
                    S.nst = std::numeric_limits<Real>::infinity();
                    S.lnamp0 = G.lnamp0[s];
                    S.v0 = G.vtx[s][0]; S.v1 = G.vtx[s][1]; S.v2 = G.vtx[s][2];
                    S.plane = G.pcode[s] != 0;
                    S.msig = -(float)G.sigma0;
                    S.K = -1;
                    if (G.tab[s] >= 0) {
                        const DevTable<Real> &T = tabs[G.tab[s]];
                        S.K = T.K;
                        S.N0 = T.N0;
                        S.Nhi = T.Nhi;
                        S.L = T.L;
                        S.lnN_lo = (float)T.lnN_lo;
                        S.inv_dl = (float)T.inv_dl;
                    }
                    for (int k = 0; k < 4; k++) sel[(g * 4 + k) * MAX_SRC + s] = S;
                }
            }
            CU(cudaMalloc(&d_sel, nn * sizeof(SrcSel<Real>)));
            CU(cudaMemcpy(d_sel, sel.data(), nn * sizeof(SrcSel<Real>), cudaMemcpyHostToDevice));
            for (size_t g = 0; g < grids.size(); g++) grids[g].sel = d_sel + g * 4 * MAX_SRC;
        }
        CU(cudaMalloc(&d_grids, grids.size() * sizeof(GridDev<Real>)));
        CU(cudaMemcpy(d_grids, grids.data(), grids.size() * sizeof(GridDev<Real>), cudaMemcpyHostToDevice));
        CU(cudaMalloc(&d_offsets, offs.size() * sizeof(long long)));
        CU(cudaMemcpy(d_offsets, offs.data(), offs.size() * sizeof(long long), cudaMemcpyHostToDevice));
        if (total > 0xffffffffll) return fail(OOTS_E_INVAL, "%lld cells in one call (the queue holds 32-bit indices)", total);
        CU(cudaMalloc(&d_queue, (size_t)std::max(total, 1ll) * sizeof(unsigned)));
        if (nsmax <= 1) CU(cudaMalloc(&d_qrec, (size_t)std::max(total, 1ll) * queue_record_bytes<Real>()));
        CU(cudaMalloc(&d_rcache, (size_t)std::max(total, 1ll) * 3 * sizeof(Real)));
        CU(cudaMalloc(&d_qcount, 8 * sizeof(unsigned)));
        CU(cudaMemset(d_qcount, 0, 8 * sizeof(unsigned)));
        if (!jobs.empty()) {
            CU(cudaMalloc(&d_jobs, jobs.size() * sizeof(Job)));
            CU(cudaMemcpy(d_jobs, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice));
            CU(cudaMalloc(&d_items, items.size() * sizeof(TileItem)));
            CU(cudaMemcpy(d_items, items.data(), items.size() * sizeof(TileItem), cudaMemcpyHostToDevice));
            CU(cudaMalloc(&d_sync, 128));
            CU(cudaMemset(d_sync, 0, 128));
            // faces start with epoch 0 in every word (flags at 0); launches use epochs 1, 2, ...
            // The pipelined kernel publishes tagged words; the throughput kernel
            // (shape 7) plain values and a flag per tile; A1 runs the pipelined
            // kernel on shape 7's tiles.
            if (!is_tp_shape(shape) || scheme == OOTS_A1) {
                const size_t fbytes = (size_t)ntiles * 3 * FMAX * face_words<Real>() * sizeof(unsigned long long);
                CU(cudaMalloc(&d_faces, fbytes));
                CU(cudaMemset(d_faces, 0, fbytes));
            }
            if (is_tp_shape(shape)) {
                CU(cudaMalloc(&d_tpfaces, (size_t)ntiles * 3 * FMAX * tp_face_comps<Real>() * sizeof(Real)));
                CU(cudaMalloc(&d_tpflags, (size_t)ntiles * sizeof(unsigned)));
                CU(cudaMemset(d_tpflags, 0, (size_t)ntiles * sizeof(unsigned)));
            }
        }
        if (!pjobs.empty()) {
            // rows along x first (their trace kernel differs), then the rest
            std::stable_sort(pjobs.begin(), pjobs.end(), [](const PlaneJob &a, const PlaneJob &b) {
                return (a.code >> 1 != 0) < (b.code >> 1 != 0);
            });
            for (auto &P : pjobs) {
                if ((P.code >> 1) == 0) { nrow0++; threads0 += plane_job_threads(P.code, P.rows); }
                P.first = plane_threads;
                plane_threads += plane_job_threads(P.code, P.rows);
            }
            CU(cudaMalloc(&d_pjobs, pjobs.size() * sizeof(PlaneJob)));
            CU(cudaMemcpy(d_pjobs, pjobs.data(), pjobs.size() * sizeof(PlaneJob), cudaMemcpyHostToDevice));
            npjobs = (int)pjobs.size();
        }
        if (!tabs.empty()) {
            CU(cudaMalloc(&d_tabs, tabs.size() * sizeof(DevTable<Real>)));
            CU(cudaMemcpy(d_tabs, tabs.data(), tabs.size() * sizeof(DevTable<Real>), cudaMemcpyHostToDevice));
        }
        CU(prepare_sweeps<Real>());
        int nsm = c0->nsm;
        nblocks0 = sweep_occupancy<Real>(shape, 0) * nsm;
        nblocks1 = sweep_occupancy<Real>(shape, 1) * nsm;
        gen_blocks = cell_general_occupancy<Real>(nsmax) * nsm;
        // closed-form passes: 128-thread blocks for many sources (a slow cell holds up fewer others),
        // 256 for one source (cheap cells; fewer block set-ups), unless tuned
        cell_bs = c0->cell_block > 0 ? c0->cell_block : (nsmax > 1 ? 128 : 256);
        return OOTS_OK;
    }

    SweepParams<Real> params(int which) const
    {
        SweepParams<Real> P;
        P.grids = d_grids;
        P.jobs = d_jobs;
        P.items = d_items;
        P.nitems = nitems;
        P.which = which;
        P.ticket = d_sync;
        P.done = d_sync + 1;
        P.epoch = d_sync + 16;
        P.faces = d_faces;
        P.tpfaces = d_tpfaces;
        P.tpflags = d_tpflags;
        P.tabs = d_tabs;
        P.err = d_err;
        P.spin_limit = spin_limit;
        P.skip_publish = skip_publish;
        P.chunk = sweep_chunk;
        P.ngrid = (int)ctxs.size();
        P.bricks = d_bricks;
        return P;
    }

    // trace (mode 0) or A1 implicit sweep (mode 1) of every source: point
    // sources by the wavefront sweep, plane sources row by row
    int sweep(cudaStream_t s, int which, int mode)
    {
        if (nitems > 0) {
            CU(cudaMemsetAsync(d_sync, 0, 2 * sizeof(unsigned), s));   // ticket and done; the epoch persists
            if (prof) prof->mark(0);
            // the trace's input in bricks (timed with the trace)
            if (mode == 0 && brick_max > 0) {
                CU(launch_pack_nx<Real>(d_grids, (int)ctxs.size(), which, shape, brick_max, ctxs[0]->nsm, s));
                if (prof) prof->mark(OOTS_K_PACK);
                if (prof) prof->mark(0);
            }
            CU(launch_sweep<Real>(params(which), shape, mode, mode == 0 ? nblocks0 : nblocks1, s));
            if (prof) prof->mark(mode == 1 ? OOTS_K_IMPLICIT : (which == 0 ? OOTS_K_SWEEP1 : OOTS_K_SWEEP2));
        }
        if (npjobs > 0) {
            if (prof) prof->mark(0);
            CU(launch_plane<Real>(d_grids, d_pjobs, npjobs, nrow0, plane_threads, threads0, d_tabs, which, mode, s));
            if (prof) prof->mark(mode == 1 ? OOTS_K_PLANE_IMPLICIT : OOTS_K_PLANE_TRACE);
        }
        return OOTS_OK;
    }

    // use_cache: the dt pass ran earlier in this substep on the same state and columns
    int cell(cudaStream_t s, int op, bool use_cache = false)
    {
        if (prof) prof->mark(0);
        CU(launch_cell<Real>(d_grids, (int)ctxs.size(), d_offsets, total, d_tabs, op, nsmax, d_queue, d_qcount, d_qrec,
                             d_rcache, use_cache ? 1 : 0, gen_blocks, cell_bs, s));
        if (prof) prof->mark(op == OP_RATEDT ? OOTS_K_RATEDT : (op == OP_HALF ? OOTS_K_HALF : OOTS_K_FULL));
        if (op == OP_RATEDT) {
            if (nsmax <= 1) return OOTS_OK;
            // several sources: the pass that checks the step hint
            if (prof) prof->mark(0);
            CU(launch_cell<Real>(d_grids, (int)ctxs.size(), d_offsets, total, d_tabs, OP_RATEDT_VERIFY, nsmax, d_queue,
                                 d_qcount, d_qrec, d_rcache, use_cache ? 1 : 0, gen_blocks, cell_bs, s));
            if (prof) prof->mark(OOTS_K_RATEDT_VERIFY);
            return OOTS_OK;
        }
        // the cells no closed form settles, one warp each
        if (prof) prof->mark(0);
        CU(launch_cell<Real>(d_grids, (int)ctxs.size(), d_offsets, total, d_tabs, op | OP_GENERAL, nsmax, d_queue,
                             d_qcount, d_qrec, d_rcache, 0, gen_blocks, cell_bs, s));
        if (prof) prof->mark(op == OP_HALF ? OOTS_K_HALF_GENERAL : OOTS_K_FULL_GENERAL);
        return OOTS_OK;
    }

    int fin(cudaStream_t s, int stage)
    {
        if (prof) prof->mark(0);
        CU(launch_finalize<Real>(d_grids, (int)ctxs.size(), stage, d_qcount, d_tabs, s));
        if (prof) prof->mark(stage == 0 ? OOTS_K_FINAL0 : OOTS_K_FINAL1);
        return OOTS_OK;
    }

    // One substep of the scheme, entirely on the device.
    int substep(cudaStream_t s, bool fixed_dt) override
    {
        int rc;
        if (scheme == OOTS_A1) {
            const oots_ctx *c = ctxs[0];
            bool need_trace = !fixed_dt && (c->crit.K3 > 0 || c->crit.K4 > 0);
            if (need_trace) {
                if ((rc = sweep(s, 0, 0))) return rc;
                if ((rc = cell(s, OP_RATEDT))) return rc;
            } else if (!fixed_dt) {
                if ((rc = cell(s, OP_RATEDT))) return rc;     // K1 only: t_rec needs no columns
            }
            if ((rc = fin(s, 0))) return rc;
            if ((rc = sweep(s, 0, 1))) return rc;
            return fin(s, 1);
        }
        if ((rc = sweep(s, 0, 0))) return rc;
        if (!fixed_dt && (rc = cell(s, OP_RATEDT))) return rc;
        if ((rc = fin(s, 0))) return rc;
        if (scheme == OOTS_A3) {
            if ((rc = cell(s, OP_HALF, !fixed_dt))) return rc;
            if ((rc = sweep(s, 1, 0))) return rc;
            if ((rc = cell(s, OP_FULL2))) return rc;
        } else {
            if ((rc = cell(s, OP_FULL1, !fixed_dt))) return rc;
        }
        return fin(s, 1);
    }

    int phase(cudaStream_t s, int ph, bool use_cache) override
    {
        switch (ph) {
        case 0: return sweep(s, 0, 0);
        case 1: return cell(s, OP_RATEDT);
        case 2: {
            int rc = fin(s, 0);
            if (rc) return rc;
            if (scheme == OOTS_A3) return cell(s, OP_HALF, use_cache);
            if ((rc = cell(s, OP_FULL1, use_cache))) return rc;
            return fin(s, 1);
        }
        case 3: return sweep(s, 1, 0);
        case 4: {
            int rc = cell(s, OP_FULL2);
            if (rc) return rc;
            return fin(s, 1);
        }
        }
        return fail(OOTS_E_INVAL, "phase %d", ph);
    }

    int trace_for_dt(cudaStream_t s) override
    {
        int rc;
        if (scheme != OOTS_A1 || ctxs[0]->crit.K3 > 0 || ctxs[0]->crit.K4 > 0)
            if ((rc = sweep(s, 0, 0))) return rc;
        return cell(s, OP_RATEDT);
    }

    int graph_replay(cudaStream_t s, int n) override
    {
        bool fixed = ctxs[0]->crit.dt_fixed > 0;
        for (auto *c : ctxs) fixed = fixed && c->crit.dt_fixed > 0;
        if (!gexec || graph_fixed != fixed) {
            if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
            if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
            CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            int rc = substep(s, fixed);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(s, &g);
            if (rc) { if (g) cudaGraphDestroy(g); return rc; }
            if (e != cudaSuccess) return fail(OOTS_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
            graph = g;
            CU(cudaGraphInstantiate(&gexec, graph, 0));
            graph_fixed = fixed;
        }
        for (int i = 0; i < n; i++) CU(cudaGraphLaunch(gexec, s));
        return OOTS_OK;
    }
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static int check_ctx(const oots_ctx *c)
{
    if (!c) return fail(OOTS_E_INVAL, "null context");
    return OOTS_OK;
}

static int pull_state(oots_ctx *c)
{
    CU(cudaSetDevice(c->device));
    CU(cudaMemcpyAsync(&c->h_st, c->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return OOTS_OK;
}

static int push_state(oots_ctx *c)
{
    CU(cudaSetDevice(c->device));
    CU(cudaMemcpyAsync(c->d_st, &c->h_st, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return OOTS_OK;
}

static int check_device_error(oots_ctx *c)
{
    int err = 0;
    CU(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (err == DEVERR_TIMEOUT) return fail(OOTS_E_DEVICE_TIMEOUT, "a wavefront tile gave up waiting for its upstream tiles");
    if (err) return fail(OOTS_E_CUDA, "device error %d", err);
    return OOTS_OK;
}

static void drop_solo(oots_ctx *c)
{
    delete c->solo;
    c->solo = nullptr;
    c->dirty = true;
}

// Allocate the per-source column arrays and (re)build the context's own launch set.
static int prepare(oots_ctx *c)
{
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid: call oots_set_grid first");
    if (c->src.empty()) return fail(OOTS_E_STATE, "no sources: call oots_add_source first");
    if (c->scheme == OOTS_A1 && c->src.size() != 1)
        return fail(OOTS_E_UNSUPPORTED, "A1 (implicit) supports a single source, got %zu", c->src.size());
    CU(cudaSetDevice(c->device));
    int ns = (int)c->src.size();
    if (ns > c->nsrc_alloc) {
        free_dev(c->d_N1);
        free_dev(c->d_N2);
        if (cudaMalloc(&c->d_N1, (size_t)ns * c->ncell * c->rsize) != cudaSuccess ||
            cudaMalloc(&c->d_N2, (size_t)ns * c->ncell * c->rsize) != cudaSuccess) {
            free_dev(c->d_N1);
            free_dev(c->d_N2);
            c->nsrc_alloc = 0;
            cudaGetLastError();
            return fail(OOTS_E_NOMEM, "column arrays for %d sources", ns);
        }
        CU(cudaMemset(c->d_N1, 0, (size_t)ns * c->ncell * c->rsize));
        CU(cudaMemset(c->d_N2, 0, (size_t)ns * c->ncell * c->rsize));
        c->nsrc_alloc = ns;
        drop_solo(c);
    }
    // device-side criteria and source totals
    int rc = pull_state(c);
    if (rc) return rc;
    c->h_st.dt_fixed = c->crit.dt_fixed;
    c->h_st.K1 = c->crit.K1;
    c->h_st.K3 = c->crit.K3;
    c->h_st.K4 = c->crit.K4;
    double sq = 0.0;
    for (auto &s : c->src) sq += source_emission(s, c->nx, c->ny, c->nz, c->dx);
    c->h_st.sumQ = sq;
    c->h_st.cell_volume = c->dx * c->dx * c->dx;
    if ((rc = push_state(c))) return rc;
    if (!c->dirty && c->solo) return OOTS_OK;
    delete c->solo;
    c->solo = nullptr;
    std::vector<oots_ctx *> one(1, c);
    if (c->precision == OOTS_FP64) {
        auto *L = new LaunchSet<double>();
        if ((rc = L->build(one, c->shape))) { delete L; return rc; }
        c->solo = L;
    } else {
        auto *L = new LaunchSet<float>();
        if ((rc = L->build(one, c->shape))) { delete L; return rc; }
        c->solo = L;
    }
    c->dirty = false;
    return OOTS_OK;
}

// Host arrays move through a device staging buffer of doubles: one copy at the
// link's bandwidth, then the checks and the conversion to the state's
// precision run on the device (at 512^3 a host loop over the cells would
// take longer than several substeps).
__global__ void fill_kernel(void *dst, int dd, double v, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (dd == 0) ((double *)dst)[i] = v;
    else ((float *)dst)[i] = (float)v;
}

// kind 0: neutral fraction, values in [0, 1]; kind 1: density, finite and > 0.
// Records the smallest failing index.
__global__ void check_kernel(const double *v, long long n, int kind, long long *bad)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = v[i];
    const bool ok = kind == 0 ? (a >= 0.0 && a <= 1.0) : (a > 0.0 && a <= 1.7976931348623157e308);
    if (!ok) atomicMin((unsigned long long *)bad, (unsigned long long)i);
}

__global__ void convert_kernel(const void *src, int sd, void *dst, int dd, long long n)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = sd == 0 ? ((const double *)src)[i] : (double)((const float *)src)[i];
    if (dd == 0) ((double *)dst)[i] = v;
    else ((float *)dst)[i] = (float)v;
}

static unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

static int ensure_stage(oots_ctx *c)
{
    if (c->d_stage) return OOTS_OK;
    if (cudaMalloc(&c->d_stage, (size_t)c->ncell * sizeof(double)) != cudaSuccess) {
        c->d_stage = nullptr;
        cudaGetLastError();
        return fail(OOTS_E_NOMEM, "staging buffer of %lld cells", c->ncell);
    }
    return OOTS_OK;
}

// Upload a host array (checked on the device first: kind as check_kernel) or
// a uniform value into dst, in the state's precision.  *bad_out receives the
// first rejected cell (-1: none); dst is untouched when a cell is rejected.
static int to_real_upload(oots_ctx *c, void *dst, const double *src, double uniform, int kind, long long *bad_out)
{
    const int own = c->precision == OOTS_FP64 ? 0 : 1;
    *bad_out = -1;
    if (!src) {
        fill_kernel<<<blocks_for(c->ncell), 256, 0, c->stream>>>(dst, own, uniform, c->ncell);
        CU(cudaGetLastError());
        CU(cudaStreamSynchronize(c->stream));
        return OOTS_OK;
    }
    int rc = ensure_stage(c);
    if (rc) return rc;
    CU(cudaMemcpyAsync(c->d_stage, src, (size_t)c->ncell * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->d_bad, 0xff, sizeof(long long), c->stream));
    check_kernel<<<blocks_for(c->ncell), 256, 0, c->stream>>>((const double *)c->d_stage, c->ncell, kind, c->d_bad);
    CU(cudaGetLastError());
    unsigned long long bad = 0;
    CU(cudaMemcpyAsync(&bad, c->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (bad != 0xffffffffffffffffull) {
        *bad_out = (long long)bad;
        return OOTS_OK;
    }
    convert_kernel<<<blocks_for(c->ncell), 256, 0, c->stream>>>(c->d_stage, 0, dst, own, c->ncell);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->stream));
    return OOTS_OK;
}

static int download_real(oots_ctx *c, const void *srcp, double *out)
{
    if (c->precision == OOTS_FP64) {
        CU(cudaMemcpyAsync(out, srcp, (size_t)c->ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    } else {
        int rc = ensure_stage(c);
        if (rc) return rc;
        convert_kernel<<<blocks_for(c->ncell), 256, 0, c->stream>>>(srcp, 1, c->d_stage, 0, c->ncell);
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(out, c->d_stage, (size_t)c->ncell * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    CU(cudaStreamSynchronize(c->stream));
    return OOTS_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *oots_version(void) { return "oots 0.1 (sm_103a)"; }

const char *oots_last_error(const oots_ctx *) { return g_err.c_str(); }

int oots_create(oots_ctx **out, int device, int precision)
{
    if (!out) return fail(OOTS_E_INVAL, "out is NULL");
    *out = nullptr;
    if (precision != OOTS_FP64 && precision != OOTS_MIXED) return fail(OOTS_E_INVAL, "precision must be OOTS_FP64 or OOTS_MIXED");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return fail(OOTS_E_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(OOTS_E_INVAL, "device %d out of range (%d devices)", device, ndev);
    oots_ctx *c = new oots_ctx();
    c->device = device;
    c->precision = precision;
    c->rsize = rsz(precision);
    CU(cudaSetDevice(device));
    CU(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device));
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return fail(OOTS_E_CUDA, "stream creation failed");
    }
    c->stream = c->own_stream;
    if (cudaMalloc(&c->d_st, sizeof(DevState)) != cudaSuccess || cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_bad, sizeof(long long)) != cudaSuccess) {
        oots_destroy(c);
        return fail(OOTS_E_NOMEM, "device state");
    }
    memset(&c->h_st, 0, sizeof(DevState));
    c->h_st.dt_bits = 0xffffffffffffffffull;
    c->h_st.done = 1;
    CU(cudaMemcpy(c->d_st, &c->h_st, sizeof(DevState), cudaMemcpyHostToDevice));
    CU(cudaMemset(c->d_err, 0, sizeof(int)));
    *out = c;
    return OOTS_OK;
}

int oots_destroy(oots_ctx *c)
{
    if (!c) return OOTS_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    delete c->solo;
    free_dev(c->d_x);
    free_dev(c->d_n);
    free_dev(c->d_xh);
    free_dev(c->d_N1);
    free_dev(c->d_N2);
    free_dev(c->d_stage);
    void *p = c->d_st;
    free_dev(p);
    p = c->d_err;
    free_dev(p);
    p = c->d_bad;
    free_dev(p);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
    return OOTS_OK;
}

int oots_set_stream(oots_ctx *c, void *stream)
{
    if (int rc = check_ctx(c)) return rc;
    CU(cudaStreamSynchronize(c->stream));
    c->stream = stream ? (cudaStream_t)stream : c->own_stream;
    if (c->solo) drop_solo(c);   // graphs are tied to nothing, but rebuild to be safe
    return OOTS_OK;
}

int oots_reset_error(oots_ctx *c)
{
    if (int rc = check_ctx(c)) return rc;
    CU(cudaSetDevice(c->device));
    CU(cudaMemset(c->d_err, 0, sizeof(int)));
    return OOTS_OK;
}

int oots_set_grid(oots_ctx *c, int nx, int ny, int nz, double dx_cm)
{
    if (int rc = check_ctx(c)) return rc;
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(dx_cm > 0) || !std::isfinite(dx_cm))
        return fail(OOTS_E_INVAL, "grid %d x %d x %d with dx %g", nx, ny, nz, dx_cm);
    if (nx > 8192 || ny > 8192 || nz > 8192) return fail(OOTS_E_INVAL, "grid side above 8192");
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    drop_solo(c);
    free_dev(c->d_x);
    free_dev(c->d_n);
    free_dev(c->d_xh);
    free_dev(c->d_N1);
    free_dev(c->d_N2);
    free_dev(c->d_stage);
    c->nsrc_alloc = 0;
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->dx = dx_cm;
    c->ncell = (long long)nx * ny * nz;
    size_t bytes = (size_t)c->ncell * c->rsize;
    if (cudaMalloc(&c->d_x, bytes) != cudaSuccess || cudaMalloc(&c->d_xh, bytes) != cudaSuccess) {
        free_dev(c->d_x);
        free_dev(c->d_xh);
        c->ncell = 0;
        cudaGetLastError();
        return fail(OOTS_E_NOMEM, "state of %lld cells", (long long)nx * ny * nz);
    }
    c->uniform_n = true;
    c->n_uniform = 1.0;
    for (auto &s : c->src)
        for (int a = 0; a < 3; a++) {
            int n3[3] = {nx, ny, nz};
            double v = std::floor(s.pos[a] + 0.5);
            s.v[a] = (int)std::min<double>(std::max<double>(v, 0.0), n3[a]);
        }
    int rc = oots_set_neutral_fraction(c, nullptr, 1.0 - 1e-6);
    if (rc) return rc;
    memset(&c->h_st, 0, sizeof(DevState));
    c->h_st.dt_bits = 0xffffffffffffffffull;
    c->h_st.done = 1;
    return push_state(c);
}

int oots_set_density(oots_ctx *c, const double *n_H, double uniform_n)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    if (!n_H) {
        if (!(uniform_n > 0) || !std::isfinite(uniform_n)) return fail(OOTS_E_INVAL, "uniform density %g", uniform_n);
        c->uniform_n = true;
        c->n_uniform = uniform_n;
        free_dev(c->d_n);
    } else {
        if (!c->d_n && cudaMalloc(&c->d_n, (size_t)c->ncell * c->rsize) != cudaSuccess) {
            c->d_n = nullptr;
            cudaGetLastError();
            return fail(OOTS_E_NOMEM, "density array");
        }
        long long bad = -1;
        int rc = to_real_upload(c, c->d_n, n_H, 0.0, 1, &bad);
        if (rc) return rc;
        if (bad >= 0) return fail(OOTS_E_INVAL, "density %g at cell %lld", n_H[bad], bad);
        c->uniform_n = false;
    }
    drop_solo(c);
    return OOTS_OK;
}

int oots_set_neutral_fraction(oots_ctx *c, const double *x, double uniform_x)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    if (!x && !(uniform_x >= 0.0 && uniform_x <= 1.0)) return fail(OOTS_E_INVAL, "neutral fraction %g outside [0,1]", uniform_x);
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    long long bad = -1;
    int rc = to_real_upload(c, c->d_x, x, uniform_x, 0, &bad);
    if (rc) return rc;
    if (bad >= 0) return fail(OOTS_E_INVAL, "neutral fraction %g at cell %lld", x[bad], bad);
    return OOTS_OK;
}

int oots_set_physics(oots_ctx *c, double alpha_B, double sigma0, double tau0, double T)
{
    if (int rc = check_ctx(c)) return rc;
    if (!(alpha_B >= 0) || !(sigma0 > 0) || !(tau0 > 0) || !(T > 0))
        return fail(OOTS_E_INVAL, "physics alpha %g sigma0 %g tau0 %g T %g", alpha_B, sigma0, tau0, T);
    c->alpha = alpha_B;
    c->sigma0 = sigma0;
    c->tau0 = tau0;
    c->T = T;
    drop_solo(c);
    return OOTS_OK;
}

int oots_add_source(oots_ctx *c, const double pos[3], double Q, int spectrum, double T_bb, int *id)
{
    if (int rc = check_ctx(c)) return rc;
    if (!pos) return fail(OOTS_E_INVAL, "pos is NULL");
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    if (!(Q > 0) || !std::isfinite(Q)) return fail(OOTS_E_INVAL, "source rate %g", Q);
    if (spectrum != OOTS_MONO && spectrum != OOTS_BLACKBODY) return fail(OOTS_E_INVAL, "spectrum %d", spectrum);
    if (spectrum == OOTS_BLACKBODY && !(T_bb >= 1e3 && T_bb <= 1e6)) return fail(OOTS_E_INVAL, "blackbody temperature %g", T_bb);
    if ((int)c->src.size() >= MAX_SRC) return fail(OOTS_E_INVAL, "at most %d sources", (int)MAX_SRC);
    SourceH S;
    const int n3[3] = {c->nx, c->ny, c->nz};
    for (int a = 0; a < 3; a++) {
        if (!std::isfinite(pos[a])) return fail(OOTS_E_INVAL, "source position not finite");
        S.pos[a] = pos[a];
        double v = std::floor(pos[a] + 0.5);
        S.v[a] = (int)std::min<double>(std::max<double>(v, 0.0), n3[a]);
    }
    S.Q = Q;
    S.spectrum = spectrum;
    S.T = T_bb;
    if (spectrum == OOTS_BLACKBODY) host_table(1, T_bb, c->sigma0);   // build now, off the hot path
    c->src.push_back(S);
    if (id) *id = (int)c->src.size() - 1;
    drop_solo(c);
    return OOTS_OK;
}

int oots_add_plane_source(oots_ctx *c, int axis, int direction, double F, int spectrum, double T_bb, int *id)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    if (axis < 0 || axis > 2) return fail(OOTS_E_INVAL, "plane source axis %d (0..2)", axis);
    if (direction != 1 && direction != -1) return fail(OOTS_E_INVAL, "plane source direction %d (+1 or -1)", direction);
    if (!(F > 0) || !std::isfinite(F)) return fail(OOTS_E_INVAL, "plane source flux %g", F);
    if (spectrum != OOTS_MONO && spectrum != OOTS_BLACKBODY) return fail(OOTS_E_INVAL, "spectrum %d", spectrum);
    if (spectrum == OOTS_BLACKBODY && !(T_bb >= 1e3 && T_bb <= 1e6)) return fail(OOTS_E_INVAL, "blackbody temperature %g", T_bb);
    if ((int)c->src.size() >= MAX_SRC) return fail(OOTS_E_INVAL, "at most %d sources", (int)MAX_SRC);
    SourceH S;
    memset(S.pos, 0, sizeof(S.pos));
    memset(S.v, 0, sizeof(S.v));
    S.Q = F;
    S.spectrum = spectrum;
    S.T = T_bb;
    S.pcode = 1 + 2 * axis + (direction < 0 ? 1 : 0);
    if (spectrum == OOTS_BLACKBODY) host_table(1, T_bb, c->sigma0);
    c->src.push_back(S);
    if (id) *id = (int)c->src.size() - 1;
    drop_solo(c);
    return OOTS_OK;
}

int oots_clear_sources(oots_ctx *c)
{
    if (int rc = check_ctx(c)) return rc;
    c->src.clear();
    drop_solo(c);
    return OOTS_OK;
}

int oots_set_scheme(oots_ctx *c, int scheme, const oots_dtcrit *crit)
{
    if (int rc = check_ctx(c)) return rc;
    if (scheme != OOTS_A1 && scheme != OOTS_A2 && scheme != OOTS_A3) return fail(OOTS_E_INVAL, "scheme %d", scheme);
    if (crit) {
        if (!(crit->dt_fixed >= 0) || std::isnan(crit->K1) || std::isnan(crit->K3) || std::isnan(crit->K4))
            return fail(OOTS_E_INVAL, "bad criteria");
        if (!(crit->dt_fixed > 0) && !(crit->K1 > 0) && !(crit->K3 > 0) && !(crit->K4 > 0))
            return fail(OOTS_E_INVAL, "no timestep criterion and no fixed dt");
        c->crit = *crit;
    }
    c->scheme = scheme;
    drop_solo(c);
    return OOTS_OK;
}

int oots_dtcrit_preset(int id, int scheme, oots_dtcrit *out)
{
    if (!out) return fail(OOTS_E_INVAL, "out is NULL");
    if (id < 0 || id > 12) return fail(OOTS_E_INVAL, "criterion id %d (0..12)", id);
    if (scheme != OOTS_A1 && scheme != OOTS_A2 && scheme != OOTS_A3) return fail(OOTS_E_INVAL, "scheme %d", scheme);
    static const double k1[5] = {1.0, 0.3, 0.1, 0.03, 0.003};
    static const double k4[5] = {1.0, 0.5, 0.25, 0.125, 0.0625};
    static const double kq[4] = {0.5, 0.25, 0.125, 0.0625};
    memset(out, 0, sizeof(*out));
    if (id <= 4) {
        if (scheme == OOTS_A1) out->K1 = k1[id];
        else out->K4 = k4[id];
    } else if (id <= 8) {
        out->K4 = kq[id - 5];
    } else {
        out->K3 = kq[id - 9];
    }
    return OOTS_OK;
}

int oots_compute_dt(oots_ctx *c, double *dt)
{
    if (int rc = check_ctx(c)) return rc;
    if (!dt) return fail(OOTS_E_INVAL, "dt is NULL");
    if (c->batched) return fail(OOTS_E_STATE, "context is part of a batch");
    int rc = prepare(c);
    if (rc) return rc;
    if ((rc = pull_state(c))) return rc;
    c->h_st.dt_bits = 0xffffffffffffffffull;
    c->h_st.done = 0;
    if ((rc = push_state(c))) return rc;
    if ((rc = c->solo->trace_for_dt(c->stream))) return rc;
    if ((rc = check_device_error(c))) return rc;
    if ((rc = pull_state(c))) return rc;
    *dt = c->h_st.dt_bits == 0xffffffffffffffffull ? 1e300 : *(double *)&c->h_st.dt_bits;
    return OOTS_OK;
}

int oots_step(oots_ctx *c, double dt)
{
    if (int rc = check_ctx(c)) return rc;
    if (!(dt > 0) || !std::isfinite(dt)) return fail(OOTS_E_INVAL, "dt %g", dt);
    if (c->batched) return fail(OOTS_E_STATE, "context is part of a batch");
    int rc = prepare(c);
    if (rc) return rc;
    if ((rc = pull_state(c))) return rc;
    c->h_st.dt_fixed = dt;
    c->h_st.t_end = c->h_st.t + dt;
    c->h_st.done = 0;
    if ((rc = push_state(c))) return rc;
    CU(cudaSetDevice(c->device));
    if ((rc = c->solo->substep(c->stream, true))) return rc;
    if ((rc = check_device_error(c))) return rc;
    if ((rc = pull_state(c))) return rc;
    c->h_st.dt_fixed = c->crit.dt_fixed;
    // the substep advanced t by exactly dt
    return push_state(c);
}

int oots_advance(oots_ctx *c, double t_end, double *t_out, long long *nsub_out)
{
    if (int rc = check_ctx(c)) return rc;
    if (!std::isfinite(t_end)) return fail(OOTS_E_INVAL, "t_end %g", t_end);
    if (c->batched) return fail(OOTS_E_STATE, "context is part of a batch");
    int rc = prepare(c);
    if (rc) return rc;
    if ((rc = pull_state(c))) return rc;
    long long n0 = c->h_st.nsub;
    if (t_end > c->h_st.t) {
        c->h_st.t_end = t_end;
        c->h_st.done = 0;
        if ((rc = push_state(c))) return rc;
        CU(cudaSetDevice(c->device));
        int burst = 1;
        for (;;) {
            if ((rc = c->solo->graph_replay(c->stream, burst))) return rc;
            if ((rc = check_device_error(c))) return rc;
            if ((rc = pull_state(c))) return rc;
            if (c->h_st.done) break;
            if (burst < 64) burst *= 2;
        }
    }
    if (t_out) *t_out = c->h_st.t;
    if (nsub_out) *nsub_out = c->h_st.nsub - n0;
    return OOTS_OK;
}

int oots_run_substeps(oots_ctx *c, long long n, double t_end)
{
    if (int rc = check_ctx(c)) return rc;
    if (n < 0 || !std::isfinite(t_end)) return fail(OOTS_E_INVAL, "n %lld, t_end %g", n, t_end);
    if (c->batched) return fail(OOTS_E_STATE, "context is part of a batch");
    int rc = prepare(c);
    if (rc) return rc;
    if ((rc = pull_state(c))) return rc;
    c->h_st.t_end = t_end;
    c->h_st.done = (t_end > c->h_st.t) ? 0 : 1;
    if ((rc = push_state(c))) return rc;
    CU(cudaSetDevice(c->device));
    return n > 0 ? c->solo->graph_replay(c->stream, (int)n) : OOTS_OK;
}

int oots_profile_substep(oots_ctx *c, int *kinds, double *ms, int nmax, int *n_out)
{
    if (int rc = check_ctx(c)) return rc;
    if (!kinds || !ms || !n_out || nmax <= 0) return fail(OOTS_E_INVAL, "profile arguments");
    if (c->batched) return fail(OOTS_E_STATE, "context is part of a batch");
    int rc = prepare(c);
    if (rc) return rc;
    if ((rc = pull_state(c))) return rc;
    if (!(c->h_st.t_end > c->h_st.t)) c->h_st.t_end = c->h_st.t + 1e300;
    c->h_st.done = 0;
    if ((rc = push_state(c))) return rc;
    CU(cudaSetDevice(c->device));
    LaunchProfiler P;
    P.s = c->stream;
    c->solo->prof = &P;
    rc = c->solo->substep(c->stream, c->crit.dt_fixed > 0);
    c->solo->prof = nullptr;
    if (rc) return rc;
    CU(cudaStreamSynchronize(c->stream));
    if ((rc = check_device_error(c))) return rc;
    int n = 0;
    for (size_t i = 0; i + 1 < P.ev.size(); i += 2) {
        if (n >= nmax) break;
        float t = 0.0f;
        CU(cudaEventElapsedTime(&t, P.ev[i], P.ev[i + 1]));
        kinds[n] = P.kinds[i + 1];
        ms[n] = t;
        n++;
    }
    *n_out = n;
    return OOTS_OK;
}

int oots_get_neutral_fraction(oots_ctx *c, double *out)
{
    if (int rc = check_ctx(c)) return rc;
    if (!out) return fail(OOTS_E_INVAL, "out is NULL");
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    return download_real(c, c->d_x, out);
}

int oots_get_column_density(oots_ctx *c, int source, double *out)
{
    if (int rc = check_ctx(c)) return rc;
    if (!out) return fail(OOTS_E_INVAL, "out is NULL");
    if (source < 0 || source >= (int)c->src.size()) return fail(OOTS_E_INVAL, "source %d", source);
    if (!c->d_N1 || source >= c->nsrc_alloc) return fail(OOTS_E_STATE, "no trace yet");
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    return download_real(c, (const char *)c->d_N1 + (size_t)source * c->ncell * c->rsize, out);
}

int oots_get_budget(oots_ctx *c, oots_budget *out)
{
    if (int rc = check_ctx(c)) return rc;
    if (!out) return fail(OOTS_E_INVAL, "out is NULL");
    int rc = pull_state(c);
    if (rc) return rc;
    out->emitted = c->h_st.bud_total[0];
    out->absorbed = c->h_st.bud_total[1];
    out->ions = c->h_st.bud_total[2];
    out->recombinations = c->h_st.bud_total[3];
    return OOTS_OK;
}

int oots_reset_budget(oots_ctx *c)
{
    if (int rc = check_ctx(c)) return rc;
    int rc = pull_state(c);
    if (rc) return rc;
    for (int q = 0; q < 4; q++) c->h_st.bud_total[q] = 0.0;
    return push_state(c);
}

int oots_get_time(oots_ctx *c, double *t, long long *nsub)
{
    if (int rc = check_ctx(c)) return rc;
    int rc = pull_state(c);
    if (rc) return rc;
    if (t) *t = c->h_st.t;
    if (nsub) *nsub = c->h_st.nsub;
    return OOTS_OK;
}

int oots_set_time(oots_ctx *c, double t)
{
    if (int rc = check_ctx(c)) return rc;
    if (!std::isfinite(t)) return fail(OOTS_E_INVAL, "t %g", t);
    int rc = pull_state(c);
    if (rc) return rc;
    c->h_st.t = t;
    return push_state(c);
}

int oots_set_neutral_fraction_device(oots_ctx *c, const void *x_dev, int dtype)
{
    if (int rc = check_ctx(c)) return rc;
    if (!x_dev || (dtype != 0 && dtype != 1)) return fail(OOTS_E_INVAL, "x_dev / dtype");
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    CU(cudaSetDevice(c->device));
    int own = c->precision == OOTS_FP64 ? 0 : 1;
    convert_kernel<<<(unsigned)((c->ncell + 255) / 256), 256, 0, c->stream>>>(x_dev, dtype, c->d_x, own, c->ncell);
    CU(cudaGetLastError());
    return OOTS_OK;
}

int oots_get_neutral_fraction_device(oots_ctx *c, void *x_dev, int dtype)
{
    if (int rc = check_ctx(c)) return rc;
    if (!x_dev || (dtype != 0 && dtype != 1)) return fail(OOTS_E_INVAL, "x_dev / dtype");
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    CU(cudaSetDevice(c->device));
    int own = c->precision == OOTS_FP64 ? 0 : 1;
    convert_kernel<<<(unsigned)((c->ncell + 255) / 256), 256, 0, c->stream>>>(c->d_x, own, x_dev, dtype, c->ncell);
    CU(cudaGetLastError());
    return OOTS_OK;
}

int oots_synchronize(oots_ctx *c)
{
    if (int rc = check_ctx(c)) return rc;
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int oots_set_tile_shape(oots_ctx *c, int shape)
{
    if (int rc = check_ctx(c)) return rc;
    if (shape < -1 || shape >= NUM_SHAPES) return fail(OOTS_E_INVAL, "tile shape %d", shape);
    c->shape = shape;
    drop_solo(c);
    return OOTS_OK;
}

int oots_tile_shape_info(int shape, int dims[3])
{
    if (shape < 0 || shape >= NUM_SHAPES) return fail(OOTS_E_INVAL, "tile shape %d", shape);
    if (dims)
        for (int a = 0; a < 3; a++) dims[a] = SHAPE_DIMS[shape][a];
    return NUM_SHAPES;
}

int oots_debug_set(oots_ctx *c, int key, long long value)
{
    if (int rc = check_ctx(c)) return rc;
    if (key == 1) {
        if (value <= 0) return fail(OOTS_E_INVAL, "spin limit %lld", value);
        c->spin_limit = value;
    } else if (key == 2) {
        c->skip_publish = value;
    } else if (key == 3) {
        if (value < 0 || value > 64) return fail(OOTS_E_INVAL, "sweep chunk %lld", value);
        c->sweep_chunk = (int)value;
    } else if (key == 4) {
        if (value != 0 && value != 1) return fail(OOTS_E_INVAL, "tile alignment %lld", value);
        c->tile_align = (int)value;
    } else if (key == 5) {
        if (value != 0 && value != 128 && value != 256) return fail(OOTS_E_INVAL, "cell block %lld", value);
        c->cell_block = (int)value;
    } else {
        return fail(OOTS_E_INVAL, "debug key %d", key);
    }
    drop_solo(c);
    return OOTS_OK;
}

// ---------------------------------------------------------------------------
// partitioned runs (one process per GPU)
// ---------------------------------------------------------------------------
int oots_set_partition(oots_ctx *c, unsigned long long src_mask, int z0, int z1)
{
    if (int rc = check_ctx(c)) return rc;
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    if (z0 < 0 || z0 > c->nz || (z1 > 0 && z1 < z0)) return fail(OOTS_E_INVAL, "z-range [%d, %d)", z0, z1);
    c->part_src = src_mask;
    c->part_z0 = z0;
    c->part_z1 = z1;
    c->phase_dt = false;
    drop_solo(c);
    return OOTS_OK;
}

int oots_run_phase(oots_ctx *c, int phase, double *value)
{
    if (int rc = check_ctx(c)) return rc;
    if (phase < OOTS_PH_TRACE1 || phase > OOTS_PH_FULL) return fail(OOTS_E_INVAL, "phase %d", phase);
    if (c->batched) return fail(OOTS_E_STATE, "context is part of a batch");
    if (c->scheme == OOTS_A1) return fail(OOTS_E_UNSUPPORTED, "phases run the explicit schemes A2 and A3");
    for (auto &S : c->src)
        if (S.pcode) return fail(OOTS_E_UNSUPPORTED, "phases take point sources only");
    if ((phase == OOTS_PH_STEP1 || phase == OOTS_PH_DT) && !value) return fail(OOTS_E_INVAL, "value is NULL");
    if (phase == OOTS_PH_FULL && c->scheme != OOTS_A3) return fail(OOTS_E_INVAL, "A2 completes in OOTS_PH_STEP1");
    if (phase == OOTS_PH_TRACE2 && c->scheme != OOTS_A3) return fail(OOTS_E_INVAL, "A2 has one trace");
    int rc = prepare(c);
    if (rc) return rc;
    CU(cudaSetDevice(c->device));
    if ((rc = pull_state(c))) return rc;
    if (phase == OOTS_PH_DT) {
        c->h_st.dt_bits = 0xffffffffffffffffull;
        c->h_st.done = 0;
    } else if (phase == OOTS_PH_STEP1) {
        const double dt = *value;
        if (!(dt > 0) || !std::isfinite(dt)) return fail(OOTS_E_INVAL, "dt %g", dt);
        c->h_st.dt_fixed = dt;
        c->h_st.t_end = c->h_st.t + dt;
        c->h_st.done = 0;
    } else {
        c->h_st.done = 0;
        if (!(c->h_st.t_end > c->h_st.t)) c->h_st.t_end = c->h_st.t + 1e300;
    }
    if ((rc = push_state(c))) return rc;
    const bool use_cache = phase == OOTS_PH_STEP1 && c->phase_dt;
    if ((rc = c->solo->phase(c->stream, phase, use_cache))) return rc;
    if ((rc = check_device_error(c))) return rc;
    if ((rc = pull_state(c))) return rc;
    if (phase == OOTS_PH_TRACE1) c->phase_dt = false;
    if (phase == OOTS_PH_DT) {
        *value = c->h_st.dt_bits == 0xffffffffffffffffull ? 1e300 : *(double *)&c->h_st.dt_bits;
        c->phase_dt = true;
    }
    if (phase == OOTS_PH_STEP1) c->phase_dt = false;
    if ((phase == OOTS_PH_STEP1 && c->scheme == OOTS_A2) || phase == OOTS_PH_FULL) {
        c->h_st.dt_fixed = c->crit.dt_fixed;
        return push_state(c);
    }
    return OOTS_OK;
}

int oots_array_device(oots_ctx *c, int kind, int source, void **ptr, unsigned long long *bytes)
{
    if (int rc = check_ctx(c)) return rc;
    if (!ptr) return fail(OOTS_E_INVAL, "ptr is NULL");
    if (c->ncell == 0) return fail(OOTS_E_STATE, "no grid");
    const size_t nb = (size_t)c->ncell * c->rsize;
    char *base = nullptr;
    if (kind == 0) base = (char *)c->d_x;
    else if (kind == 1) base = (char *)c->d_xh;
    else if (kind == 2 || kind == 3) {
        if (source < 0 || source >= (int)c->src.size()) return fail(OOTS_E_INVAL, "source %d", source);
        int rc = prepare(c);                 // the column arrays exist once the context is prepared
        if (rc) return rc;
        base = (char *)(kind == 2 ? c->d_N1 : c->d_N2) + (size_t)source * nb;
    } else {
        return fail(OOTS_E_INVAL, "array kind %d", kind);
    }
    *ptr = base;
    if (bytes) *bytes = nb;
    return OOTS_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
struct oots_batch {
    std::vector<oots_ctx *> ctxs;
    LaunchSetBase *L = nullptr;
    cudaStream_t stream = nullptr;
};

int oots_batch_create(oots_batch **out, oots_ctx *const *ctxs, int n)
{
    if (!out || !ctxs || n <= 0) return fail(OOTS_E_INVAL, "batch arguments");
    *out = nullptr;
    if (n > 65535) return fail(OOTS_E_INVAL, "%d contexts in one batch (at most 65535)", n);
    for (int i = 0; i < n; i++) {
        if (!ctxs[i]) return fail(OOTS_E_INVAL, "context %d is NULL", i);
        if (ctxs[i]->device != ctxs[0]->device || ctxs[i]->precision != ctxs[0]->precision)
            return fail(OOTS_E_INVAL, "batched contexts must share device and precision");
        if (ctxs[i]->scheme != ctxs[0]->scheme || ctxs[i]->scheme == OOTS_A1)
            return fail(OOTS_E_UNSUPPORTED, "batched contexts must share scheme A2 or A3");
        if ((ctxs[i]->crit.dt_fixed > 0) != (ctxs[0]->crit.dt_fixed > 0))
            return fail(OOTS_E_INVAL, "batched contexts must all use fixed or all adaptive dt");
        if (ctxs[i]->batched) return fail(OOTS_E_STATE, "context %d already in a batch", i);
        int rc = prepare(ctxs[i]);
        if (rc) return rc;
    }
    oots_batch *b = new oots_batch();
    b->ctxs.assign(ctxs, ctxs + n);
    b->stream = ctxs[0]->stream;
    int rc;
    if (ctxs[0]->precision == OOTS_FP64) {
        auto *L = new LaunchSet<double>();
        if ((rc = L->build(b->ctxs, ctxs[0]->shape))) { delete L; delete b; return rc; }
        b->L = L;
    } else {
        auto *L = new LaunchSet<float>();
        if ((rc = L->build(b->ctxs, ctxs[0]->shape))) { delete L; delete b; return rc; }
        b->L = L;
    }
    for (auto *c : b->ctxs) c->batched = true;
    *out = b;
    return OOTS_OK;
}

int oots_batch_advance(oots_batch *b, const double *t_end_each, long long *nsub_out)
{
    if (!b || !t_end_each) return fail(OOTS_E_INVAL, "batch arguments");
    std::vector<long long> n0(b->ctxs.size());
    bool any = false;
    for (size_t i = 0; i < b->ctxs.size(); i++) {
        oots_ctx *c = b->ctxs[i];
        int rc = pull_state(c);
        if (rc) return rc;
        n0[i] = c->h_st.nsub;
        if (t_end_each[i] > c->h_st.t) {
            c->h_st.t_end = t_end_each[i];
            c->h_st.done = 0;
            any = true;
        } else {
            c->h_st.done = 1;
        }
        if ((rc = push_state(c))) return rc;
    }
    if (any) {
        CU(cudaSetDevice(b->ctxs[0]->device));
        int burst = 1;
        for (;;) {
            int rc = b->L->graph_replay(b->stream, burst);
            if (rc) return rc;
            if ((rc = check_device_error(b->ctxs[0]))) return rc;
            bool all = true;
            for (auto *c : b->ctxs) {
                if ((rc = pull_state(c))) return rc;
                all = all && c->h_st.done;
            }
            if (all) break;
            if (burst < 64) burst *= 2;
        }
    }
    if (nsub_out)
        for (size_t i = 0; i < b->ctxs.size(); i++) nsub_out[i] = b->ctxs[i]->h_st.nsub - n0[i];
    return OOTS_OK;
}

int oots_batch_run_substeps(oots_batch *b, long long n, const double *t_end_each)
{
    if (!b || !t_end_each || n < 0) return fail(OOTS_E_INVAL, "batch arguments");
    for (size_t i = 0; i < b->ctxs.size(); i++) {
        if (!std::isfinite(t_end_each[i])) return fail(OOTS_E_INVAL, "t_end %g of context %zu", t_end_each[i], i);
        oots_ctx *c = b->ctxs[i];
        int rc = pull_state(c);
        if (rc) return rc;
        c->h_st.t_end = t_end_each[i];
        c->h_st.done = (t_end_each[i] > c->h_st.t) ? 0 : 1;
        if ((rc = push_state(c))) return rc;
    }
    CU(cudaSetDevice(b->ctxs[0]->device));
    return n > 0 ? b->L->graph_replay(b->stream, (int)n) : OOTS_OK;
}

int oots_batch_destroy(oots_batch *b)
{
    if (!b) return OOTS_OK;
    if (!b->ctxs.empty()) {
        cudaSetDevice(b->ctxs[0]->device);
        cudaStreamSynchronize(b->stream);
    }
    for (auto *c : b->ctxs) c->batched = false;
    delete b->L;
    delete b;
    return OOTS_OK;
}

} // extern "C"
