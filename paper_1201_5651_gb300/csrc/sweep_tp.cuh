// Throughput form of the short-characteristics sweep (Mackey 2012, Sect. 2:
// columns by short characteristics with the Mellema et al. 2006 weighting;
// Sect. 5: octants traced outward from the source vertex independently).
//
// When many sources or grids share a launch, tiles are plentiful and the
// wavefront's depth no longer sets the pace: the per-cell instruction count,
// the memory latency each tile waits through and the tiles each SM keeps in
// flight do.  This kernel trades the pipelined kernel's early hand-off for a
// lean tile: TX x 8 x 8 cells (TX = 8 or 16), 64 threads, no producer or
// writer warps, and a shared-memory footprint small enough for 9-16 tiles per
// SM.  A tile waits for its whole upstream halo, sweeps, then publishes its
// three downstream faces as plain values (12 bytes per face cell in the mixed
// path, half the pipelined kernel's tagged words) followed by one flag per
// tile, set with release semantics to the launch's epoch; a downstream tile
// acquires the flags of its upstream tiles before it reads their faces.  The
// two kernels share the work list.
//
// Inside an octant, a cell takes its entry column from the upwind layer of its
// dominant axis only.  Wherever one axis dominates every cell of a tile (all
// tiles off the octant's diagonal planes i = j, j = k, i = k), the tile is
// therefore swept layer by layer along that axis, every thread busy at each
// step (one or two cells of the layer).  The other tiles hold tied cells,
// which average the interpolations along their tied axes; they are swept
// plane by plane (i + j + k) with one thread per (j,k) column.
//
// Included by sweep_impl.cuh ahead of the launch wrappers.
#pragma once

namespace oots {

// Shared-memory layout of a throughput tile with its one-cell upstream halo:
// index (lk+1) SZ + (lj+1) SY + (li+1).  The strides were chosen by counting
// bank conflicts over the access patterns of the passes (cell loads, the
// three layer orientations, the diagonal planes): at most two-way.
template <int TX> struct TpLayout {
    static constexpr int TY = 8, TZ = 8;
    static constexpr int SY = TX == 8 ? 9 : 18;
    static constexpr int SZ = TX == 8 ? 88 : 169;
    static constexpr int HSZ = (TZ + 1) * SZ;
    static constexpr int NT = TY * TZ;                 // threads
    static constexpr int NC = TX * TY * TZ;            // cells
    static constexpr int NP = TX + TY + TZ - 2;        // planes i + j + k of a tile
    static constexpr OOTS_HD int h(int li, int lj, int lk) { return (lk + 1) * SZ + (lj + 1) * SY + (li + 1); }
    static_assert(TY * SY + TX < SZ, "rows fit below the next plane");
    static_assert(HSZ < (1 << 14), "halo entry packing");
};

// The halo and face lists of a tile in the pipelined kernel's packing, with
// the throughput layout's shared-memory index in the low 14 bits.  Unlike the
// pipelined kernel's lists (sorted by the plane that first needs an entry),
// these keep the faces' own order, so that a warp's 32 entries are adjacent
// in the published face and its loads and stores touch whole sectors.
template <int TX> struct TpLists {
    unsigned halo[TileLayout<TX, 8, 8>::NE];
    unsigned face[FaceList<TX, 8, 8>::N];
};
template <int TX> constexpr unsigned tp_repack(unsigned e)
{
    typedef TileLayout<TX, 8, 8> P;
    const int hp = (int)(e & 0x3fffu);
    const int li = hp % P::SZ % P::SY - 1, lj = hp % P::SZ / P::SY - 1, lk = hp / P::SZ - 1;
    return (e & ~0x3fffu) | (unsigned)TpLayout<TX>::h(li, lj, lk);
}
template <int TX> constexpr TpLists<TX> make_tp_lists()
{
    TpLists<TX> R{};
    for (int q = 0; q < TileLayout<TX, 8, 8>::NE; q++) {
        int key = 0; unsigned p = 0;
        halo_entry<TX, 8, 8>(q, key, p);
        R.halo[q] = tp_repack<TX>(p);
    }
    for (int q = 0; q < FaceList<TX, 8, 8>::N; q++) {
        int key = 0; unsigned p = 0;
        face_entry<TX, 8, 8>(q, key, p);
        R.face[q] = tp_repack<TX>(p);
    }
    return R;
}
template <int TX> __device__ const TpLists<TX> g_tp_lists = make_tp_lists<TX>();

template <typename Real, int TX> constexpr size_t sweep_tp_smem()
{
    return (size_t)TpLayout<TX>::HSZ * (sizeof(typename ColT<Real>::type) + 2 * sizeof(Real));
}

// Entry column of a cell with octant indices idx at halo index h, from the
// N_out and weight factors W = 1/max(dtau, tau0) of its upwind neighbours:
// for each tied dominant axis a, the bilinear weights of the entry point on
// the upwind layer (c_t/c_a for the t-1 neighbour) times W, normalised; the
// tied axes' interpolations are averaged.  Neighbours outside the octant are
// dropped.  Written as weighted differences to one reference neighbour, so
// the float-float column is not rounded to float before the increment.  The
// reference is the neighbour one step back along every tied axis, which
// always carries weight (with three tied axes all of it): a neighbour that
// carries none would make the result a difference of columns far larger
// than itself near the source vertex.
template <typename Real, int TX>
__device__ __forceinline__ typename ColT<Real>::type
sc_entry_general(const typename ColT<Real>::type *sN, const Real *sW, int h, const int idx[3])
{
    typedef TpLayout<TX> L;
    const int str[3] = {1, L::SY, L::SZ};
    const int c2[3] = {2 * idx[0] + 1, 2 * idx[1] + 1, 2 * idx[2] + 1};
    const int cm = max(c2[0], max(c2[1], c2[2]));
    if (cm == 1) return ColT<Real>::zero();                 // the cell at the vertex
    const int sref = (c2[0] == cm ? str[0] : 0) + (c2[1] == cm ? str[1] : 0) + (c2[2] == cm ? str[2] : 0);
    const typename ColT<Real>::type Nref = sN[h - sref];
    const Real inv_nt = Real(1) / Real((c2[0] == cm) + (c2[1] == cm) + (c2[2] == cm));
    Real d = Real(0);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (c2[a] != cm) continue;
        const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
        const int ha = h - str[a], s1 = str[t1], s2 = str[t2];
        const Real w1 = Real(c2[t1]) / Real(c2[a]);
        const Real w2 = Real(c2[t2]) / Real(c2[a]);
        Real wv[4], dv[4], ws = Real(0);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int e1 = e & 1, e2 = e >> 1;
            const bool ok = idx[t1] - e1 >= 0 && idx[t2] - e2 >= 0;
            const int hn = ha - (e1 ? s1 : 0) - (e2 ? s2 : 0);
            wv[e] = ok ? (e1 ? w1 : Real(1) - w1) * (e2 ? w2 : Real(1) - w2) * sW[hn] : Real(0);
            dv[e] = ok ? ColT<Real>::sub_r(sN[hn], Nref) : Real(0);
            ws += wv[e];
        }
        if (ws > Real(0)) d += inv_nt / ws * (wv[0] * dv[0] + wv[1] * dv[1] + wv[2] * dv[2] + wv[3] * dv[3]);
    }
    return ColT<Real>::add(Nref, d);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Start fetching `bytes` (a multiple of 16, 16-byte aligned) into L2, without waiting.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Reciprocal and square root: correctly rounded in FP64, the fast
// approximations in the mixed path (a few ulp; the mixed path is judged on its
// error against FP64).
__device__ __forceinline__ double tp_rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float tp_rcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double tp_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float tp_sqrt(float a) { return a * rsqrtf(a); }   // a > 0 here

// Entry column of a cell with one dominant axis: bilinear weights of the
// entry point on the upwind layer (g1 = c_t1/c_a for the t1-1 neighbour,
// g2 for t2-1) times the neighbours' factors W (0 outside the octant),
// normalised; weighted differences to the (0,0) neighbour at h00.
template <typename Real>
__device__ __forceinline__ typename ColT<Real>::type
sc_entry_axis(const typename ColT<Real>::type *sN, const Real *sW, int h00, int s1, int s2, Real g1, Real g2)
{
    const Real w00 = (Real(1) - g1) * (Real(1) - g2) * sW[h00];
    const Real w01 = (Real(1) - g1) * g2 * sW[h00 - s2];
    const Real w10 = g1 * (Real(1) - g2) * sW[h00 - s1];
    const Real w11 = g1 * g2 * sW[h00 - s1 - s2];
    const typename ColT<Real>::type N00 = sN[h00];
    const Real d = (w01 * ColT<Real>::sub_r(sN[h00 - s2], N00) + w10 * ColT<Real>::sub_r(sN[h00 - s1], N00) +
                    w11 * ColT<Real>::sub_r(sN[h00 - s1 - s2], N00)) *
                   tp_rcp(w00 + w01 + w10 + w11);
    return ColT<Real>::add(N00, d);
}

// The trace's input n x (density times neutral fraction of the traced state)
// in bricks of TX x 8 x 8 cells, x fastest within a brick and bricks x
// fastest (zero outside the grid).  Tiles start at global multiples of the
// tile, so each tile of each octant lies in one brick and reads its cells as
// one contiguous block, where the grid's own layout gives it 64 rows of TX
// cells in two arrays.  The product is rounded as the sweep would round it.
// One row of blocks per grid (blockIdx.y).
template <typename Real, int TX>
__global__ void __launch_bounds__(256) pack_nx_kernel(const GridDev<Real> *grids, int which)
{
    const GridDev<Real> &G = grids[blockIdx.y];
    Real *B = G.nxb;
    if (B == nullptr) return;
    constexpr unsigned NC = TX * 64u;
    if (G.st->done) return;                          // past its end time: nothing is traced
    const Real *xs = which == 1 ? G.xh : G.x;
    const Real *n = G.n;
    const Real nu = G.n_uniform;
    const unsigned nbx = (unsigned)G.nbx, nbxy = (unsigned)G.nbx * (unsigned)G.nby;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long long total = (long long)nbxy * (unsigned)G.nbz * NC;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const unsigned b = (unsigned)(q / NC), e = (unsigned)(q % NC);
        const int gi = (int)(b % nbx) * TX + (int)(e % TX);
        const int gj = (int)(b % nbxy / nbx) * 8 + (int)(e / TX % 8);
        const int gk = (int)(b / nbxy) * 8 + (int)(e / (TX * 8));
        Real v = Real(0);
        if (gi < nx && gj < ny && gk < nz) {
            const long long g = gi + (long long)nx * (gj + (long long)ny * gk);
            v = (n ? __ldg(n + g) : nu) * __ldg(xs + g);
        }
        B[q] = v;
    }
}

// four consecutive values (16-byte aligned for float, 32 for double)
__device__ __forceinline__ void tp_load4(const float *p, float v[4])
{
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void tp_load4(const double *p, double v[4])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// compile-time constants passed to the kernel's generic lambdas
template <int V> struct TpInt { static constexpr int value = V; };

template <typename Real, int TX>
__global__ void __launch_bounds__(64, sizeof(Real) == 4 ? (TX == 8 ? 16 : 9) : 8) sweep_tp_kernel(SweepParams<Real> P)
{
    typedef typename ColT<Real>::type Col;
    typedef TpLayout<TX> L;
    constexpr int NT = L::NT, HSZ = L::HSZ;
    constexpr int SY = L::SY, SZ = L::SZ;
    constexpr int FMAX = (TX * 8 > 64) ? TX * 8 : 64;   // largest face of the tile
    constexpr int NCOMP = tp_face_comps<Real>();
    constexpr int NQ = TX / 8;                          // cells per thread in a layer across x
    static_assert(NT == 64, "64 threads: one per (j,k) column");
    typedef TileLayout<TX, 8, 8> HL_L;                 // the packed lists' tile
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Col *sN = reinterpret_cast<Col *>(smem_raw);      // N_out
    Real *sW = reinterpret_cast<Real *>(sN + HSZ);     // 1/max(dtau, tau0); 0 outside the octant
    Real *sDI = sW + HSZ;                              // increment n x ds, then N_in
    __shared__ unsigned s_next;                        // the CTA's next ticket (claimed one tile ahead)
    __shared__ int s_bad;
    const TpLists<TX> &TL = g_tp_lists<TX>;
    const unsigned epoch = *(volatile unsigned *)P.epoch + 1u;
    const int tid = threadIdx.x;
    const int c8 = tid % 8, r8 = tid / 8;             // (j,k) column of this thread

    if (tid == 0) s_next = sweep_live(P) ? atomicAdd(P.ticket, 1u) : (unsigned)P.nitems;
    __syncthreads();
    for (;;) {
        const unsigned tk = s_next;
        if (tk >= (unsigned)P.nitems) break;
        const TileItem it = P.items[tk];
        if (P.ngrid > 1 && P.grids[it.grid].st->done) {
            // a grid past its end time skips every tile (all of them, so no wait is left pending);
            // with one grid the launch returned at once instead
            __syncthreads();
            if (tid == 0) s_next = atomicAdd(P.ticket, 1u);
            __syncthreads();
            continue;
        }
        const Job J = P.jobs[it.job];
        const GridDev<Real> &G = P.grids[J.grid];
        const int o0[3] = {it.I * TX - J.off[0], it.J * 8 - J.off[1], it.K * 8 - J.off[2]};
        const long long tile_self = J.tile_base + ((long long)it.K * J.nt[1] + it.J) * J.nt[0] + it.I;
        const Real *xin = (P.which == 1) ? G.xh : G.x;
        const Real dx = G.dx, sig = G.sigma0, tau0 = G.tau0;
        const long long sx = 1, sy = J.nt[0], sz = (long long)J.nt[0] * J.nt[1];
        const unsigned have = (it.I > 0 ? 1u : 0u) | (it.J > 0 ? 2u : 0u) | (it.K > 0 ? 4u : 0u);

        // 1. the upstream tiles (up to seven: the three face neighbours and the
        //    four edge and corner ones): wait until each has published in this
        //    launch (bounded); the halo is read after the barrier below
        if (tid == 0) s_bad = 0;
        __syncthreads();
        if (tid >= 1 && tid <= 7 && (tid & ~have) == 0) {
            const long long up = tile_self - ((tid & 1) ? sx : 0) - ((tid & 2) ? sy : 0) - ((tid & 4) ? sz : 0);
            long long spins = 0;
            unsigned ns = 32;
            while (ld_acquire_u32(P.tpflags + up) != epoch) {
                if (++spins > P.spin_limit) { atomicCAS(P.err, 0, (int)DEVERR_TIMEOUT); s_bad = 1; break; }
                if ((spins & 31) == 0 && *(volatile int *)P.err != 0) { s_bad = 1; break; }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
            }
        }
        // the next ticket, claimed now so that it is back by the halo step
        unsigned tk_next = 0u;
        if (tid == 0) tk_next = atomicAdd(P.ticket, 1u);
        // 2. own cells: increments n x ds and weight factors.  Cell e = tid + 64 u
        //    (x fastest); the global index moves by fixed strides (octant signs
        //    folded in), four cells' loads in flight at a time.
        const long long sxg = J.sg[0], syg = (long long)J.sg[1] * G.nx, szg = (long long)J.sg[2] * G.nx * G.ny;
        const long long gbase = (long long)(J.sg[0] > 0 ? J.v[0] + o0[0] : J.v[0] - 1 - o0[0]) +
                                (long long)G.nx * ((long long)(J.sg[1] > 0 ? J.v[1] + o0[1] : J.v[1] - 1 - o0[1]) +
                                                   (long long)G.ny * (J.sg[2] > 0 ? J.v[2] + o0[2] : J.v[2] - 1 - o0[2]));
        const int i_lo = max(-o0[0], 0), i_hi = min(J.ext[0] - o0[0], TX);   // in-octant local ranges
        const int j_lo = max(-o0[1], 0), j_hi = min(J.ext[1] - o0[1], 8);
        const int k_lo = max(-o0[2], 0), k_hi = min(J.ext[2] - o0[2], 8);
        if (G.nxb != nullptr) {
            // the tile's brick (its index set with the work list); thread tid
            // takes brick cells 4 (tid + 64 v) .. +3
            const Real *brick = reinterpret_cast<const Real *>(P.bricks) + (long long)it.brick * L::NC;
#pragma unroll
            for (int v = 0; v < L::NC / 256; v++) {
                const int e0 = 4 * (tid + 64 * v);
                const int bj = (e0 / TX) % 8, bk = e0 / (TX * 8);
                const int lj = J.sg[1] > 0 ? bj : 7 - bj, lk = J.sg[2] > 0 ? bk : 7 - bk;
                const bool row_in = lj >= j_lo && lj < j_hi && lk >= k_lo && lk < k_hi;
                Real nxv[4];
                if (row_in) tp_load4(brick + e0, nxv);
                const Real c1 = Real(o0[1] + lj) + Real(0.5), c2 = Real(o0[2] + lk) + Real(0.5);
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const int bi = e0 % TX + c;
                    const int li = J.sg[0] > 0 ? bi : TX - 1 - bi;
                    const int h = L::h(li, lj, lk);
                    Real dN = Real(0), wf = Real(0);
                    if (row_in && li >= i_lo && li < i_hi) {
                        const Real c0 = Real(o0[0] + li) + Real(0.5);
                        const Real ds =
                            dx * tp_sqrt(c0 * c0 + c1 * c1 + c2 * c2) * tp_rcp(m_max(c0, m_max(c1, c2)));
                        dN = nxv[c] * ds;
                        wf = tp_rcp(m_max(sig * dN, tau0));
                    }
                    sN[h] = ColT<Real>::zero();
                    sW[h] = wf;
                    sDI[h] = dN;
                }
            }
        } else {
#pragma unroll
            for (int b = 0; b < TX; b += 4) {
                Real nv[4], xv[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int e = tid + 64 * (b + u);
                    const int li = e % TX, lj = (e / TX) % 8, lk = e / (TX * 8);
                    const bool in = li >= i_lo && li < i_hi && lj >= j_lo && lj < j_hi && lk >= k_lo && lk < k_hi;
                    const long long gq = gbase + li * sxg + lj * syg + lk * szg;
                    nv[u] = in ? (G.n ? __ldg(G.n + gq) : G.n_uniform) : Real(0);
                    xv[u] = in ? __ldg(xin + gq) : Real(0);
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int e = tid + 64 * (b + u);
                    const int li = e % TX, lj = (e / TX) % 8, lk = e / (TX * 8);
                    const int h = L::h(li, lj, lk);
                    Real dN = Real(0), wf = Real(0);
                    if (li >= i_lo && li < i_hi && lj >= j_lo && lj < j_hi && lk >= k_lo && lk < k_hi) {
                        const Real c0 = Real(o0[0] + li) + Real(0.5), c1 = Real(o0[1] + lj) + Real(0.5),
                                   c2 = Real(o0[2] + lk) + Real(0.5);
                        const Real ds = dx * tp_sqrt(c0 * c0 + c1 * c1 + c2 * c2) * tp_rcp(m_max(c0, m_max(c1, c2)));
                        dN = nv[u] * xv[u] * ds;
                        wf = tp_rcp(m_max(sig * dN, tau0));
                    }
                    sN[h] = ColT<Real>::zero();
                    sW[h] = wf;
                    sDI[h] = dN;
                }
            }
        }
        __syncthreads();
        // 3. the halo from the upstream tiles' published faces (read past L1)
        const bool bad = s_bad != 0;
        for (int q = tid; q < HL_L::NE; q += NT) {
            const unsigned en = __ldg(&TL.halo[q]);
            const unsigned mask = en >> 28;
            const int h = (int)(en & 0x3fffu);
            Col vN = ColT<Real>::zero();
            Real vW = Real(0);
            if ((mask & ~have) == 0 && !bad) {
                const long long src = tile_self - ((mask & 1) ? sx : 0) - ((mask & 2) ? sy : 0) - ((mask & 4) ? sz : 0);
                const Real *f = P.tpfaces + (src * 3 + (long long)((en >> 26) & 3u)) * NCOMP * FMAX + ((en >> 14) & 0xfffu);
                if (sizeof(Real) == 4) {
                    vN = ColT<Real>::make(__ldcg(f), __ldcg(f + FMAX));
                    vW = __ldcg(f + 2 * FMAX);
                } else {
                    vN = ColT<Real>::make(__ldcg(f), Real(0));
                    vW = __ldcg(f + FMAX);
                }
            }
            sN[h] = vN;
            sW[h] = vW;
        }
        // hand on the next ticket, and start its brick on its way into L2
        if (tid == 0) {
            s_next = tk_next;
            if (P.bricks != nullptr && tk_next < (unsigned)P.nitems)
                prefetch_l2_bulk(reinterpret_cast<const Real *>(P.bricks) +
                                     (long long)__ldg(&P.items[tk_next].brick) * L::NC,
                                 (unsigned)(L::NC * sizeof(Real)));
        }
        __syncthreads();

        // 4. one dominant axis over the whole tile (in-octant cells), or mixed
        const int lo0 = o0[0] + i_lo, lo1 = o0[1] + j_lo, lo2 = o0[2] + k_lo;
        const int hi0 = o0[0] + i_hi - 1, hi1 = o0[1] + j_hi - 1, hi2 = o0[2] + k_hi - 1;
        int pure = -1;
        if (lo0 > hi1 && lo0 > hi2) pure = 0;
        else if (lo1 > hi0 && lo1 > hi2) pure = 1;
        else if (lo2 > hi0 && lo2 > hi1) pure = 2;

        // Layer by layer along the dominant axis a, the axis fixed at compile
        // time (the halo strides become immediate offsets).
        // a = 0: this thread's cell (l, c8, r8), transverse t1 = y, t2 = z;
        // a = 1 (t1 = z, t2 = x) and a = 2 (t1 = x, t2 = y): cells (li, lb) with
        // lb the other transverse index, li = tid % TX, lb = tid / TX + q 64/TX.
        auto layers = [&](auto A_) {
            constexpr int a = decltype(A_)::value;
            constexpr int sa = a == 0 ? 1 : (a == 1 ? SY : SZ);
            constexpr int s1 = a == 0 ? SY : (a == 1 ? SZ : 1);
            constexpr int s2 = a == 0 ? SZ : (a == 1 ? 1 : SY);
            if constexpr (a == 0) {
                const int lj = c8, lk = r8;
                const bool col_in = lj >= j_lo && lj < j_hi && lk >= k_lo && lk < k_hi;
                const Real c1 = Real(2 * (o0[1] + lj) + 1), c2 = Real(2 * (o0[2] + lk) + 1);
                for (int l = 0; l < TX; l++) {
                    if (col_in && l >= i_lo && l < i_hi) {
                        const int h = L::h(l, lj, lk);
                        const Real ica = tp_rcp(Real(2 * (o0[0] + l) + 1));
                        const Col Nin = sc_entry_axis<Real>(sN, sW, h - sa, s1, s2, c1 * ica, c2 * ica);
                        sN[h] = ColT<Real>::add(Nin, sDI[h]);
                        sDI[h] = ColT<Real>::to_real(Nin);
                    }
                    __syncthreads();
                }
            } else {
                const int oa = a == 1 ? o0[1] : o0[2];
                const int ob = a == 1 ? o0[2] : o0[1];
                const int la_lo = a == 1 ? j_lo : k_lo, la_hi = a == 1 ? j_hi : k_hi;
                const int lb_lo = a == 1 ? k_lo : j_lo, lb_hi = a == 1 ? k_hi : j_hi;
                const int li = tid % TX;
                const bool i_in = li >= i_lo && li < i_hi;
                const Real cx = Real(2 * (o0[0] + li) + 1);
                for (int l = 0; l < 8; l++) {
                    if (l >= la_lo && l < la_hi && i_in) {
                        const Real ica = tp_rcp(Real(2 * (oa + l) + 1));
#pragma unroll
                        for (int q = 0; q < NQ; q++) {
                            const int lb = tid / TX + q * (64 / TX);
                            if (lb >= lb_lo && lb < lb_hi) {
                                const int h = a == 1 ? L::h(li, l, lb) : L::h(li, lb, l);
                                const Real cb = Real(2 * (ob + lb) + 1);
                                // a = 1: g1 for the z-1 neighbour, g2 for x-1; a = 2: g1 for x-1, g2 for y-1
                                const Real g1 = (a == 1 ? cb : cx) * ica, g2 = (a == 1 ? cx : cb) * ica;
                                const Col Nin = sc_entry_axis<Real>(sN, sW, h - sa, s1, s2, g1, g2);
                                sN[h] = ColT<Real>::add(Nin, sDI[h]);
                                sDI[h] = ColT<Real>::to_real(Nin);
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        };
        if (pure >= 0) {
            if (pure == 0) layers(TpInt<0>{});
            else if (pure == 1) layers(TpInt<1>{});
            else layers(TpInt<2>{});
        } else {
            // plane by plane (li + lj + lk = m), one thread per (lj, lk) column;
            // cells with one dominant axis take the cheap form, tied cells the
            // average over their tied axes, the vertex cell N_in = 0
            const int lj = c8, lk = r8;
            const int j = o0[1] + lj, k = o0[2] + lk;
            const bool col_in = lj >= j_lo && lj < j_hi && lk >= k_lo && lk < k_hi;
            for (int m = 0; m < L::NP; m++) {
                const int li = m - lj - lk;
                if (col_in && li >= i_lo && li < i_hi) {
                    const int i = o0[0] + li;
                    const int h = L::h(li, lj, lk);
                    const int c2i = 2 * i + 1, c2j = 2 * j + 1, c2k = 2 * k + 1;
                    const int cm = max(c2i, max(c2j, c2k));
                    const int ntied = (c2i == cm) + (c2j == cm) + (c2k == cm);
                    Col Nin;
                    if (ntied == 1) {
                        const int a = c2i == cm ? 0 : (c2j == cm ? 1 : 2);
                        const int sa = a == 0 ? 1 : (a == 1 ? SY : SZ);
                        const int s1 = a == 0 ? SY : (a == 1 ? SZ : 1);
                        const int s2 = a == 0 ? SZ : (a == 1 ? 1 : SY);
                        const int ct1 = a == 0 ? c2j : (a == 1 ? c2k : c2i);
                        const int ct2 = a == 0 ? c2k : (a == 1 ? c2i : c2j);
                        const Real ica = tp_rcp(Real(cm));
                        Nin = sc_entry_axis<Real>(sN, sW, h - sa, s1, s2, Real(ct1) * ica, Real(ct2) * ica);
                    } else {
                        const int idx[3] = {i, j, k};
                        Nin = sc_entry_general<Real, TX>(sN, sW, h, idx);
                    }
                    sN[h] = ColT<Real>::add(Nin, sDI[h]);
                    sDI[h] = ColT<Real>::to_real(Nin);
                }
                __syncthreads();
            }
        }

        // 5. entry columns of the tile's cells, then its downstream faces and flag
        Real *Nout = (P.which == 1 ? G.N2 : G.N1) + (long long)J.src * G.ncell;
#pragma unroll 4
        for (int u = 0; u < TX; u++) {
            const int e = tid + 64 * u;
            const int li = e % TX, lj = (e / TX) % 8, lk = e / (TX * 8);
            if (li >= i_lo && li < i_hi && lj >= j_lo && lj < j_hi && lk >= k_lo && lk < k_hi)
                Nout[gbase + li * sxg + lj * syg + lk * szg] = sDI[L::h(li, lj, lk)];
        }
        if (tile_self != P.skip_publish) {
            Real *fbase = P.tpfaces + tile_self * 3 * NCOMP * FMAX;
            for (int q = tid; q < FaceList<TX, 8, 8>::N; q += NT) {
                const unsigned en = __ldg(&TL.face[q]);
                const int h = (int)(en & 0x3fffu);
                Real *f = fbase + ((en >> 26) & 3u) * NCOMP * FMAX + ((en >> 14) & 0xfffu);
                const Col v = sN[h];
                if (sizeof(Real) == 4) {
                    __stcg(f, ColT<Real>::hi(v));
                    __stcg(f + FMAX, ColT<Real>::lo(v));
                    __stcg(f + 2 * FMAX, sW[h]);
                } else {
                    __stcg(f, ColT<Real>::hi(v));
                    __stcg(f + FMAX, sW[h]);
                }
            }
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                st_release_u32(P.tpflags + tile_self, epoch);
            }
        }
        __syncthreads();
    }
    // the last CTA to finish advances the epoch for the next launch
    if (tid == 0 && atomicAdd(P.done, 1u) == gridDim.x - 1) *(volatile unsigned *)P.epoch = epoch;
}

} // namespace oots
