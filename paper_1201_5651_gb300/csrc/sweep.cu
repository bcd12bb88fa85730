// Short-characteristics wavefront sweep (Mackey 2012, Sect. 2: column
// densities from point sources by short characteristics with the Mellema et
// al. 2006 optical-depth weighting; Sect. 5: the source sits on a cell vertex
// and each octant is traced outward independently).
//
// GB300 layout: one persistent launch covers every (grid, source, octant) of
// the call.  The octants are cut into tiles of TX x TY x TZ cells aligned to
// global multiples of the tile size (coalesced rows).  Tiles are handed out by
// an atomic ticket in order of their tile diagonal I+J+K, so every upstream
// tile was claimed by a running CTA before any tile that waits for it.  A CTA
//   1. loads its cells' x and n (before waiting: this overlaps the wait) and
//      forms each cell's column increment n x ds and weight factor
//      1/max(dtau, tau0);
//   2. waits (bounded spin, acquire) for the three face-adjacent upstream
//      tiles; edge and corner neighbours are complete by transitivity;
//   3. gathers its one-cell halo from their published faces;
//   4. runs the plane-by-plane recurrence i+j+k = m in shared memory, one
//      thread per (j, k) column of the tile;
//   5. publishes its three downstream faces (release) and then writes the
//      entry columns of its cells to global memory.
// The recurrence is linear in the columns with weights fixed by the state, so
// only the weighted sum and one add sit on the critical path of a plane.
#include "common.cuh"
#include "integrator.cuh"
#include "kernels.h"

namespace oots {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename Col> __device__ __forceinline__ Col ld_face(const Col *p);
template <> __device__ __forceinline__ double ld_face<double>(const double *p) { return __ldcg(p); }
template <> __device__ __forceinline__ ff ld_face<ff>(const ff *p)
{
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return ff{v.x, v.y};
}

template <typename Real, int TX, int TY, int TZ, int MODE>
__global__ void __launch_bounds__(TY *TZ)
sweep_kernel(SweepParams<Real> P)
{
    typedef typename ColT<Real>::type Col;
    constexpr int HX = TX + 1, HY = TY + 1, HZ = TZ + 1;
    constexpr int NT = TY * TZ;
    constexpr int NC = TX * TY * TZ;
    constexpr int FMAX = (TY * TZ > TX * TZ ? (TY * TZ > TX * TY ? TY * TZ : TX * TY) : (TX * TZ > TX * TY ? TX * TZ : TX * TY));
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Col *sN = reinterpret_cast<Col *>(smem_raw);                       // N_out, halo-indexed
    Real *sW = reinterpret_cast<Real *>(sN + HZ * HY * HX);            // 1/max(dtau, tau0); 0 outside the octant
    Real *sD = sW + HZ * HY * HX;                                      // column increment n x ds (MODE 1: x0)
    Real *sI = sD + NC;                                                // entry column N_in (output)
    Real *sG1 = sI + NC;                                               // 1-D weight of the t1-1 neighbour
    Real *sG2 = sG1 + NC;                                              // 1-D weight of the t2-1 neighbour
    unsigned char *sMode = reinterpret_cast<unsigned char *>(sG2 + NC); // per-cell chain mode (see below)
    __shared__ unsigned s_ticket;
    __shared__ double s_bud[3];

    Col *const faceN = reinterpret_cast<Col *>(P.faceN_raw);
    const int tid = threadIdx.x;
    const int clj = tid % TY, clk = tid / TY;
    double bud_ions = 0.0, bud_rec = 0.0;
    int bud_grid = -1;

    auto hidx = [](int li, int lj, int lk) { return ((lk + 1) * HY + (lj + 1)) * HX + (li + 1); };

    for (;;) {
        if (tid == 0) {
            unsigned t = atomicAdd(P.ticket, 1u);
            // a grid that has reached its end time skips every tile (all its
            // tiles skip, so no wait is left pending)
            if (t < (unsigned)P.nitems && P.grids[P.jobs[P.items[t].job].grid].st->done) t |= 0x80000000u;
            s_ticket = t;
        }
        __syncthreads();
        const unsigned tk = s_ticket;
        if ((tk & 0x7fffffffu) >= (unsigned)P.nitems) break;
        if (tk & 0x80000000u) { __syncthreads(); continue; }
        const unsigned t = tk;
        const TileItem it = P.items[t];
        const Job J = P.jobs[it.job];
        const GridDev<Real> &G = P.grids[J.grid];
        const int i0 = it.I * TX - J.off[0], j0 = it.J * TY - J.off[1], k0 = it.K * TZ - J.off[2];
        const long long tile_self = J.tile_base + ((long long)it.K * J.nt[1] + it.J) * J.nt[0] + it.I;
        const Real *xin = (P.which == 1) ? G.xh : G.x;
        const Real dx = G.dx, sig = G.sigma0, tau0 = G.tau0;

        // 1. own cells: increments and weight factors (halo entries zeroed)
        for (int e = tid; e < HZ * HY * HX; e += NT) { sW[e] = Real(0); sN[e] = ColT<Real>::zero(); }
        __syncthreads();
        for (int e = tid; e < NC; e += NT) {
            const int li = e % TX, lj = (e / TX) % TY, lk = e / (TX * TY);
            const int i = i0 + li, j = j0 + lj, k = k0 + lk;
            Real dN = Real(0);
            // chain mode: bits 0-1 dominant axis; bit 2 / bit 3: the t1-1 / t2-1
            // neighbour exists (inside the octant); bit 4 the vertex cell; bit 5
            // tied dominant axis (general path); bit 7 outside the octant
            unsigned char mode = 0x80;
            if (i >= 0 && j >= 0 && k >= 0 && i < J.ext[0] && j < J.ext[1] && k < J.ext[2]) {
                const int c2i[3] = {2 * i + 1, 2 * j + 1, 2 * k + 1};
                const int idx3[3] = {i, j, k};
                const int cmi = max(c2i[0], max(c2i[1], c2i[2]));
                const int nt = (c2i[0] == cmi) + (c2i[1] == cmi) + (c2i[2] == cmi);
                if (i + j + k == 0) mode = 0x10;
                else if (nt > 1) mode = 0x20;
                else {
                    const int a = c2i[0] == cmi ? 0 : (c2i[1] == cmi ? 1 : 2);
                    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
                    mode = (unsigned char)(a | (idx3[t1] > 0 ? 4 : 0) | (idx3[t2] > 0 ? 8 : 0));
                    sG1[e] = Real(c2i[t1]) / Real(c2i[a]);
                    sG2[e] = Real(c2i[t2]) / Real(c2i[a]);
                }
                const int X = J.sg[0] > 0 ? J.v[0] + i : J.v[0] - 1 - i;
                const int Y = J.sg[1] > 0 ? J.v[1] + j : J.v[1] - 1 - j;
                const int Z = J.sg[2] > 0 ? J.v[2] + k : J.v[2] - 1 - k;
                const long long g = (long long)X + (long long)G.nx * ((long long)Y + (long long)G.ny * Z);
                const Real n = G.n ? __ldg(G.n + g) : G.n_uniform;
                const Real xv = __ldg(xin + g);
                const Real c0 = Real(i) + Real(0.5), c1 = Real(j) + Real(0.5), c2 = Real(k) + Real(0.5);
                const Real cm = m_max(c0, m_max(c1, c2));
                const Real ds = dx * m_sqrt(c0 * c0 + c1 * c1 + c2 * c2) / cm;
                if (MODE == 0) {
                    dN = n * xv * ds;
                    sW[hidx(li, lj, lk)] = Real(1) / m_max(sig * dN, tau0);
                } else {
                    dN = xv;                               // A1: x0, integrated in the chain
                    sW[hidx(li, lj, lk)] = Real(1);        // set in the chain
                }
            }
            sD[e] = dN;
            sMode[e] = mode;
        }

        // 2. wait for the face-adjacent upstream tiles
        if (tid == 0) {
            long long up[3];
            int nup = 0;
            if (it.I > 0) up[nup++] = tile_self - 1;
            if (it.J > 0) up[nup++] = tile_self - J.nt[0];
            if (it.K > 0) up[nup++] = tile_self - (long long)J.nt[0] * J.nt[1];
            for (int q = 0; q < nup; q++) {
                long long spins = 0;
                unsigned ns = 32;
                while (ld_acquire(P.flags + up[q]) == 0u) {
                    if (++spins > P.spin_limit) { atomicCAS(P.err, 0, (int)DEVERR_TIMEOUT); break; }
                    __nanosleep(ns);
                    if (ns < 1024) ns <<= 1;
                }
            }
        }
        __syncthreads();

        // 3. halo from the published faces
        {
            const long long sx = 1, sy = J.nt[0], sz = (long long)J.nt[0] * J.nt[1];
            // li = -1 plane (X faces of tiles I-1, with J-1 / K-1 edges)
            for (int q = tid; q < HY * HZ; q += NT) {
                const int lj = q % HY - 1, lk = q / HY - 1;
                if (it.I == 0 || (lj < 0 && it.J == 0) || (lk < 0 && it.K == 0)) continue;
                const long long src = tile_self - sx - (lj < 0 ? sy : 0) - (lk < 0 ? sz : 0);
                const int fq = (lk < 0 ? TZ - 1 : lk) * TY + (lj < 0 ? TY - 1 : lj);
                const long long o = src * 3 * FMAX + 0 * FMAX + fq;
                sN[hidx(-1, lj, lk)] = ld_face<Col>(faceN + o);
                sW[hidx(-1, lj, lk)] = __ldcg(P.faceW + o);
            }
            // lj = -1 plane (Y faces of tiles J-1, with K-1 edge)
            for (int q = tid; q < TX * HZ; q += NT) {
                const int li = q % TX, lk = q / TX - 1;
                if (it.J == 0 || (lk < 0 && it.K == 0)) continue;
                const long long src = tile_self - sy - (lk < 0 ? sz : 0);
                const int fq = (lk < 0 ? TZ - 1 : lk) * TX + li;
                const long long o = src * 3 * FMAX + 1 * FMAX + fq;
                sN[hidx(li, -1, lk)] = ld_face<Col>(faceN + o);
                sW[hidx(li, -1, lk)] = __ldcg(P.faceW + o);
            }
            // lk = -1 plane (Z face of tile K-1)
            for (int q = tid; q < TX * TY; q += NT) {
                const int li = q % TX, lj = q / TX;
                if (it.K == 0) continue;
                const long long o = (tile_self - sz) * 3 * FMAX + 2 * FMAX + lj * TX + li;
                sN[hidx(li, lj, -1)] = ld_face<Col>(faceN + o);
                sW[hidx(li, lj, -1)] = __ldcg(P.faceW + o);
            }
        }
        __syncthreads();

        // 4. plane-by-plane recurrence
        for (int m = 0; m < TX + TY + TZ - 2; m++) {
            const int li = m - clj - clk;
            if (tid < NT && li >= 0 && li < TX) {
                const int lj = clj, lk = clk;
                const int i = i0 + li, j = j0 + lj, k = k0 + lk;
                const int e = (lk * TY + lj) * TX + li;
                const unsigned mode = sMode[e];
                if (!(mode & 0x80)) {
                    const int idx[3] = {i, j, k};
                    const int loc[3] = {li, lj, lk};
                    const int c2[3] = {2 * i + 1, 2 * j + 1, 2 * k + 1};
                    const int cm = max(c2[0], max(c2[1], c2[2]));
                    Col Nin = ColT<Real>::zero();
                    if (!(mode & 0x30)) {
                        // one dominant axis a: bilinear weights of the four upwind
                        // cells times their optical-depth factors, normalised once
                        const int a = mode & 3;
                        const int str[3] = {1, HX, HX * HY};
                        const int s1 = str[a == 2 ? 0 : a + 1], s2 = str[a == 0 ? 2 : a - 1];   // strides of t1, t2
                        const int h00 = hidx(li, lj, lk) - str[a];
                        const Real g1 = sG1[e], g2 = sG2[e];
                        const Real w00 = (Real(1) - g1) * (Real(1) - g2) * sW[h00];
                        const Real w01 = (mode & 8) ? (Real(1) - g1) * g2 * sW[h00 - s2] : Real(0);
                        const Real w10 = (mode & 4) ? g1 * (Real(1) - g2) * sW[h00 - s1] : Real(0);
                        const Real w11 = ((mode & 12) == 12) ? g1 * g2 * sW[h00 - s1 - s2] : Real(0);
                        const Real r = Real(1) / (w00 + w01 + w10 + w11);
                        Col acc = ColT<Real>::fma_w(ColT<Real>::zero(), w00 * r, sN[h00]);
                        if (mode & 8) acc = ColT<Real>::fma_w(acc, w01 * r, sN[h00 - s2]);
                        if (mode & 4) acc = ColT<Real>::fma_w(acc, w10 * r, sN[h00 - s1]);
                        if ((mode & 12) == 12) acc = ColT<Real>::fma_w(acc, w11 * r, sN[h00 - s1 - s2]);
                        Nin = acc;
                    } else if (mode & 0x20) {
                        Col sum = ColT<Real>::zero();
                        int ntied = 0;
#pragma unroll
                        for (int a = 0; a < 3; a++) {
                            if (c2[a] != cm) continue;
                            ntied++;
                            const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
                            const Real w1 = Real(c2[t1]) / Real(c2[a]);   // weight of the t1-1 neighbour
                            const Real w2 = Real(c2[t2]) / Real(c2[a]);
                            Col acc = ColT<Real>::zero();
                            Real ws = Real(0);
#pragma unroll
                            for (int e1 = 0; e1 < 2; e1++) {
#pragma unroll
                                for (int e2 = 0; e2 < 2; e2++) {
                                    if (idx[t1] - e1 < 0 || idx[t2] - e2 < 0) continue;
                                    int nb[3];
                                    nb[a] = loc[a] - 1;
                                    nb[t1] = loc[t1] - e1;
                                    nb[t2] = loc[t2] - e2;
                                    const int h = hidx(nb[0], nb[1], nb[2]);
                                    const Real wg = (e1 ? w1 : Real(1) - w1) * (e2 ? w2 : Real(1) - w2);
                                    const Real w = wg * sW[h];
                                    acc = ColT<Real>::fma_w(acc, w, sN[h]);
                                    ws += w;
                                }
                            }
                            if (ws > Real(0)) sum = ColT<Real>::addc(sum, ColT<Real>::div(acc, ws));
                        }
                        Nin = ColT<Real>::div(sum, Real(ntied));
                    }
                    const Real nin_r = ColT<Real>::to_real(Nin);
                    sI[e] = nin_r;
                    if (MODE == 0) {
                        sN[hidx(li, lj, lk)] = ColT<Real>::add(Nin, sD[e]);
                    } else {
                        // A1 (Eq. 3): integrate the cell with its entry column
                        // frozen; pass on N_in - ln<f>/sigma0
                        const int X = J.sg[0] > 0 ? J.v[0] + i : J.v[0] - 1 - i;
                        const int Y = J.sg[1] > 0 ? J.v[1] + j : J.v[1] - 1 - j;
                        const int Z = J.sg[2] > 0 ? J.v[2] + k : J.v[2] - 1 - k;
                        const long long g = (long long)X + (long long)G.nx * ((long long)Y + (long long)G.ny * Z);
                        const Real n = G.n ? __ldg(G.n + g) : G.n_uniform;
                        const Real c0 = Real(i) + Real(0.5), c1 = Real(j) + Real(0.5), c2r = Real(k) + Real(0.5);
                        const Real r2 = c0 * c0 + c1 * c1 + c2r * c2r;
                        const Real cmr = m_max(c0, m_max(c1, c2r));
                        const Real sf = m_sqrt(r2) / cmr;
                        SrcRate<Real> r;
                        const int s = J.src;
                        r.Nin = nin_r;
                        r.tab = G.tab[s];
                        if (r.tab < 0) {
                            r.A = G.qfac[s] * m_exp(-sig * nin_r) / (n * r2 * sf);
                            r.b = sig * n * dx * sf;
                            r.p = Real(1);
                        } else {
                            r.A = G.qfac[s] / (n * r2 * sf);
                            r.b = n * dx * sf;
                            r.p = m_exp(tab_lnp(P.tabs[r.tab], nin_r));
                        }
                        CellODE<Real> C;
                        C.ns = 1; C.c = G.alpha * n; C.b0 = sig * n * dx * sf; C.r = &r; C.tabs = P.tabs;
                        const Real dt = Real(G.st->dt);
                        IntResult<Real> R = integrate_cell<Real, 1>(C, sD[e], dt, sig);
                        Real dtau_eff = -R.lnfav;
                        if (!(dtau_eff >= Real(0))) dtau_eff = Real(0);
                        sN[hidx(li, lj, lk)] = ColT<Real>::add(Nin, dtau_eff / sig);
                        sW[hidx(li, lj, lk)] = Real(1) / m_max(dtau_eff, tau0);
                        if (dt > Real(0)) {
                            G.xout[g] = R.x;
                            const double nV = double(n) * G.st->cell_volume;
                            bud_ions += nV * double(sD[e] - R.x);
                            bud_rec += nV * double(R.IR);
                            bud_grid = J.grid;
                        }
                    }
                }
            }
            __syncthreads();
        }

        // 5. publish the downstream faces, then write the entry columns
        {
            const long long base = tile_self * 3 * FMAX;
            for (int q = tid; q < TY * TZ; q += NT) {
                const int lj = q % TY, lk = q / TY;
                const int h = hidx(TX - 1, lj, lk);
                faceN[base + 0 * FMAX + q] = sN[h];
                P.faceW[base + 0 * FMAX + q] = sW[h];
            }
            for (int q = tid; q < TX * TZ; q += NT) {
                const int li = q % TX, lk = q / TX;
                const int h = hidx(li, TY - 1, lk);
                faceN[base + 1 * FMAX + q] = sN[h];
                P.faceW[base + 1 * FMAX + q] = sW[h];
            }
            for (int q = tid; q < TX * TY; q += NT) {
                const int li = q % TX, lj = q / TX;
                const int h = hidx(li, lj, TZ - 1);
                faceN[base + 2 * FMAX + q] = sN[h];
                P.faceW[base + 2 * FMAX + q] = sW[h];
            }
        }
        __syncthreads();
        if (tid == 0 && tile_self != P.skip_publish) {
            __threadfence();
            st_release(P.flags + tile_self, 1u);
        }
        {
            Real *Nout = (P.which == 1 ? G.N2 : G.N1) + (long long)J.src * G.ncell;
            for (int e = tid; e < NC; e += NT) {
                const int li = e % TX, lj = (e / TX) % TY, lk = e / (TX * TY);
                const int i = i0 + li, j = j0 + lj, k = k0 + lk;
                if (i >= 0 && j >= 0 && k >= 0 && i < J.ext[0] && j < J.ext[1] && k < J.ext[2]) {
                    const int X = J.sg[0] > 0 ? J.v[0] + i : J.v[0] - 1 - i;
                    const int Y = J.sg[1] > 0 ? J.v[1] + j : J.v[1] - 1 - j;
                    const int Z = J.sg[2] > 0 ? J.v[2] + k : J.v[2] - 1 - k;
                    const long long g = (long long)X + (long long)G.nx * ((long long)Y + (long long)G.ny * Z);
                    Nout[g] = sI[e];
                }
            }
        }
        __syncthreads();
    }

    if (MODE == 1) {
        // photon budget of the implicit sweep: block sums, one atomic per block
        if (tid == 0) { s_bud[0] = 0.0; s_bud[1] = 0.0; }
        __syncthreads();
        if (bud_grid >= 0) {
            atomicAdd(&s_bud[0], bud_ions);
            atomicAdd(&s_bud[1], bud_rec);
        }
        __syncthreads();
        if (tid == 0 && (s_bud[0] != 0.0 || s_bud[1] != 0.0)) {
            DevState *st = P.grids[0].st;
            atomicAdd(&st->bud_step[2], s_bud[0]);
            atomicAdd(&st->bud_step[3], s_bud[1]);
            atomicAdd(&st->bud_step[1], s_bud[0] + s_bud[1]);
        }
    }
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
template <typename Real, int TX, int TY, int TZ>
constexpr size_t sweep_smem()
{
    return (size_t)(TX + 1) * (TY + 1) * (TZ + 1) * (sizeof(typename ColT<Real>::type) + sizeof(Real))
         + (size_t)4 * TX * TY * TZ * sizeof(Real) + (size_t)TX * TY * TZ;
}

template <typename Real, int TX, int TY, int TZ, int MODE>
static cudaError_t launch_shape(const SweepParams<Real> &P, int nblocks, cudaStream_t s)
{
    constexpr size_t sm = sweep_smem<Real, TX, TY, TZ>();
    sweep_kernel<Real, TX, TY, TZ, MODE><<<nblocks, TY * TZ, sm, s>>>(P);
    return cudaGetLastError();
}

// Largest dynamic shared memory a block may use on this device.
static int max_optin_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

template <typename Real, int TX, int TY, int TZ, int MODE>
static cudaError_t prepare_shape()
{
    constexpr size_t sm = sweep_smem<Real, TX, TY, TZ>();
    if ((int)sm > max_optin_smem()) return cudaSuccess;     // shape unavailable at this precision
    return cudaFuncSetAttribute(sweep_kernel<Real, TX, TY, TZ, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
}

template <typename Real>
bool sweep_shape_ok(int shape)
{
    size_t sm = 0;
#define OOTS_SM(ID, TX, TY, TZ) if (shape == ID) sm = sweep_smem<Real, TX, TY, TZ>();
    OOTS_SHAPES(OOTS_SM)
#undef OOTS_SM
    return sm > 0 && (int)sm <= max_optin_smem();
}
template bool sweep_shape_ok<double>(int);
template bool sweep_shape_ok<float>(int);

template <typename Real>
int sweep_occupancy(int shape, int mode)
{
    int nb = 0;
    cudaError_t e = cudaSuccess;
#define OOTS_OCC(ID, TX, TY, TZ)                                                                      \
    if (shape == ID) {                                                                                \
        constexpr size_t sm = sweep_smem<Real, TX, TY, TZ>();                                         \
        if (mode == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<Real, TX, TY, TZ, 0>, TY * TZ, sm); \
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<Real, TX, TY, TZ, 1>, TY * TZ, sm); \
    }
    OOTS_SHAPES(OOTS_OCC)
#undef OOTS_OCC
    if (e != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

template <typename Real>
cudaError_t launch_sweep(const SweepParams<Real> &P, int shape, int mode, int nblocks, cudaStream_t s)
{
    if (P.nitems <= 0) return cudaSuccess;
    long long nb = nblocks;
    if (nb > P.nitems) nb = P.nitems;
    if (nb < 1) nb = 1;
#define OOTS_LAUNCH(ID, TX, TY, TZ)                                                         \
    if (shape == ID) {                                                                      \
        return mode == 0 ? launch_shape<Real, TX, TY, TZ, 0>(P, (int)nb, s)                 \
                         : launch_shape<Real, TX, TY, TZ, 1>(P, (int)nb, s);                \
    }
    OOTS_SHAPES(OOTS_LAUNCH)
#undef OOTS_LAUNCH
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t prepare_sweeps()
{
    cudaError_t e = cudaSuccess, e2;
#define OOTS_PREP(ID, TX, TY, TZ)                                  \
    e2 = prepare_shape<Real, TX, TY, TZ, 0>(); if (e2 != cudaSuccess) e = e2; \
    e2 = prepare_shape<Real, TX, TY, TZ, 1>(); if (e2 != cudaSuccess) e = e2;
    OOTS_SHAPES(OOTS_PREP)
#undef OOTS_PREP
    return e;
}

template int sweep_occupancy<double>(int, int);
template int sweep_occupancy<float>(int, int);
template cudaError_t prepare_sweeps<double>();
template cudaError_t prepare_sweeps<float>();
template cudaError_t launch_sweep<double>(const SweepParams<double> &, int, int, int, cudaStream_t);
template cudaError_t launch_sweep<float>(const SweepParams<float> &, int, int, int, cudaStream_t);

} // namespace oots
