// Throughput form of the short-characteristics sweep (Mackey 2012, Sect. 2:
// columns by short characteristics with the Mellema et al. 2006 weighting;
// Sect. 5: octants traced outward from the source vertex independently).
//
// When many sources or grids share a launch, tiles are plentiful and the
// wavefront's depth no longer sets the pace: the per-cell instruction count
// and the warps each SM keeps busy do.  This kernel trades the pipelined
// kernel's early hand-off for a lean tile: T x T x T cells (T = 8), T^2
// threads, no producer or writer warps, and a shared-memory footprint small
// enough for about sixteen tiles per SM.  A tile waits for its whole upstream
// halo, sweeps, then publishes its three downstream faces in the same tagged
// words as the pipelined kernel (the two kernels share the work list and the
// face buffers).
//
// Inside an octant, a cell takes its entry column from the upwind layer of its
// dominant axis only.  Wherever one axis dominates every cell of a tile (all
// tiles off the octant's diagonal planes i = j, j = k, i = k), the tile is
// therefore swept layer by layer along that axis, with one thread per cell of
// the layer: T steps, every thread busy at each.  The other tiles hold tied
// cells, which average the interpolations along their tied axes; they are
// swept plane by plane (i + j + k) with one thread per (j,k) column.
//
// Included by sweep_impl.cuh ahead of the launch wrappers.
#pragma once

namespace oots {

// Shared-memory layout of a throughput tile with its one-cell upstream halo:
// index (lk+1) SZ + (lj+1) SY + (li+1).  The strides keep a layer's accesses
// (lanes over two of the three axes) free of bank conflicts for two of the
// three layer orientations and at most two-way for the third.
template <int T> struct TpLayout {
    static constexpr int SY = T + 1;
    static constexpr int SZ = T == 8 ? 88 : (T + 1) * (T + 1);
    static constexpr int HSZ = (T + 1) * SZ;
    static constexpr int NT = T * T;
    static constexpr int NP = 3 * T - 2;
    static constexpr OOTS_HD int h(int li, int lj, int lk) { return (lk + 1) * SZ + (lj + 1) * SY + (li + 1); }
    static_assert(T * SY + T < SZ, "rows fit below the next plane");
    static_assert(HSZ < (1 << 14), "halo entry packing");
};

template <typename Real, int T> constexpr size_t sweep_tp_smem()
{
    return (size_t)TpLayout<T>::HSZ * (sizeof(typename ColT<Real>::type) + 2 * sizeof(Real));
}

// Entry column of a cell with octant indices idx at halo index h, from the
// N_out and weight factors W = 1/max(dtau, tau0) of its upwind neighbours:
// for each tied dominant axis a, the bilinear weights of the entry point on
// the upwind layer (c_t/c_a for the t-1 neighbour) times W, normalised; the
// tied axes' interpolations are averaged.  Neighbours outside the octant are
// dropped.  Written as weighted differences to one reference neighbour, so
// the float-float column is not rounded to float before the increment.
template <typename Real, int T>
__device__ __forceinline__ typename ColT<Real>::type
sc_entry_general(const typename ColT<Real>::type *sN, const Real *sW, int h, const int idx[3])
{
    typedef TpLayout<T> L;
    const int str[3] = {1, L::SY, L::SZ};
    const int c2[3] = {2 * idx[0] + 1, 2 * idx[1] + 1, 2 * idx[2] + 1};
    const int cm = max(c2[0], max(c2[1], c2[2]));
    if (cm == 1) return ColT<Real>::zero();                 // the cell at the vertex
    const int sref = c2[0] == cm ? str[0] : (c2[1] == cm ? str[1] : str[2]);   // first tied axis
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

template <typename Real, int T>
__global__ void __launch_bounds__(T *T) sweep_tp_kernel(SweepParams<Real> P)
{
    typedef typename ColT<Real>::type Col;
    typedef TpLayout<T> L;
    constexpr int NT = L::NT, NC = T * T * T, HSZ = L::HSZ;
    constexpr int SY = L::SY, SZ = L::SZ;
    constexpr int FMAX = T * T;
    typedef TileLayout<T, T, T> HL_L;                 // layout the halo and face lists are packed for
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Col *sN = reinterpret_cast<Col *>(smem_raw);      // N_out
    Real *sW = reinterpret_cast<Real *>(sN + HSZ);     // 1/max(dtau, tau0); 0 outside the octant
    Real *sDI = sW + HSZ;                              // increment n x ds, then N_in
    __shared__ unsigned s_ticket;
    const HaloList<T, T, T> &HL = g_halo_list<T, T, T>;
    const FaceList<T, T, T> &FL = g_face_list<T, T, T>;
    typedef FaceWords<Real> FW;
    unsigned long long *const faces = P.faces;
    const unsigned epoch = *(volatile unsigned *)P.epoch + 1u;
    const int tid = threadIdx.x;
    const int tu = tid % T, tv = tid / T;              // this thread's cell within a layer or column

    // halo index of the packed halo/face list entries (packed for the pipelined layout)
    auto remap = [](unsigned hp) {
        const int li = (int)(hp % HL_L::SZ % HL_L::SY) - 1;
        const int lj = (int)(hp % HL_L::SZ / HL_L::SY) - 1;
        const int lk = (int)(hp / HL_L::SZ) - 1;
        return L::h(li, lj, lk);
    };

    for (;;) {
        if (tid == 0) {
            unsigned t = atomicAdd(P.ticket, 1u);
            if (t < (unsigned)P.nitems && P.grids[P.jobs[P.items[t].job].grid].st->done) t |= 0x80000000u;
            s_ticket = t;
        }
        __syncthreads();
        const unsigned tk = s_ticket;
        if ((tk & 0x7fffffffu) >= (unsigned)P.nitems) break;
        if (tk & 0x80000000u) { __syncthreads(); continue; }
        const TileItem it = P.items[tk];
        const Job J = P.jobs[it.job];
        const GridDev<Real> &G = P.grids[J.grid];
        const int o0[3] = {it.I * T - J.off[0], it.J * T - J.off[1], it.K * T - J.off[2]};
        const long long tile_self = J.tile_base + ((long long)it.K * J.nt[1] + it.J) * J.nt[0] + it.I;
        const Real *xin = (P.which == 1) ? G.xh : G.x;
        const Real dx = G.dx, sig = G.sigma0, tau0 = G.tau0;

        // 1. own cells: increments n x ds and weight factors (four loads in flight per thread)
        for (int e0 = tid; e0 < NC; e0 += 4 * NT) {
            long long gq[4];
            bool in[4];
            Real nv[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int e = e0 + u * NT;
                const int li = e % T, lj = (e / T) % T, lk = e / (T * T);
                const int i = o0[0] + li, j = o0[1] + lj, k = o0[2] + lk;
                in[u] = e < NC && i >= 0 && j >= 0 && k >= 0 && i < J.ext[0] && j < J.ext[1] && k < J.ext[2];
                const int X = J.sg[0] > 0 ? J.v[0] + i : J.v[0] - 1 - i;
                const int Y = J.sg[1] > 0 ? J.v[1] + j : J.v[1] - 1 - j;
                const int Z = J.sg[2] > 0 ? J.v[2] + k : J.v[2] - 1 - k;
                gq[u] = (long long)X + (long long)G.nx * ((long long)Y + (long long)G.ny * Z);
                nv[u] = in[u] ? (G.n ? __ldg(G.n + gq[u]) : G.n_uniform) : Real(0);
                xv[u] = in[u] ? __ldg(xin + gq[u]) : Real(0);
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int e = e0 + u * NT;
                if (e >= NC) continue;
                const int li = e % T, lj = (e / T) % T, lk = e / (T * T);
                const int h = L::h(li, lj, lk);
                Real dN = Real(0), wf = Real(0);
                if (in[u]) {
                    const Real c0 = Real(o0[0] + li) + Real(0.5), c1 = Real(o0[1] + lj) + Real(0.5),
                               c2 = Real(o0[2] + lk) + Real(0.5);
                    const Real ds = dx * m_sqrt(c0 * c0 + c1 * c1 + c2 * c2) / m_max(c0, m_max(c1, c2));
                    dN = nv[u] * xv[u] * ds;
                    wf = Real(1) / m_max(sig * dN, tau0);
                }
                sN[h] = ColT<Real>::zero();
                sW[h] = wf;
                sDI[h] = dN;
            }
        }
        // 2. the upstream halo: poll each published cell until its words carry
        //    this launch's epoch (bounded), or zero it where no upstream tile exists
        {
            const long long sx = 1, sy = J.nt[0], sz = (long long)J.nt[0] * J.nt[1];
            const unsigned have = (it.I > 0 ? 1u : 0u) | (it.J > 0 ? 2u : 0u) | (it.K > 0 ? 4u : 0u);
            for (int q = tid; q < HL_L::NE; q += NT) {
                const unsigned en = __ldg(&HL.e[q]);
                const unsigned mask = en >> 28;
                const int h = remap(en & 0x3fffu);
                Col vN = ColT<Real>::zero();
                Real vW = Real(0);
                if ((mask & ~have) == 0) {
                    const long long src = tile_self - ((mask & 1) ? sx : 0) - ((mask & 2) ? sy : 0) - ((mask & 4) ? sz : 0);
                    const long long o = ((src * 3 + (long long)((en >> 26) & 3u)) * FMAX + ((en >> 14) & 0xfffu)) * FW::W;
                    bool ok = FW::load(faces + o, epoch, vN, vW);
                    long long spins = 0;
                    unsigned ns = 32;
                    while (!ok) {
                        if (++spins > P.spin_limit) { atomicCAS(P.err, 0, (int)DEVERR_TIMEOUT); break; }
                        if ((spins & 31) == 0 && *(volatile int *)P.err != 0) break;
                        __nanosleep(ns);
                        if (ns < 256) ns <<= 1;
                        ok = FW::load(faces + o, epoch, vN, vW);
                    }
                    if (!ok) { vN = ColT<Real>::zero(); vW = Real(0); }
                }
                sN[h] = vN;
                sW[h] = vW;
            }
        }
        __syncthreads();

        // 3. one dominant axis over the whole tile (in-octant cells), or mixed
        const int lo0 = max(o0[0], 0), lo1 = max(o0[1], 0), lo2 = max(o0[2], 0);
        const int hi0 = min(o0[0] + T, J.ext[0]) - 1, hi1 = min(o0[1] + T, J.ext[1]) - 1,
                  hi2 = min(o0[2] + T, J.ext[2]) - 1;
        int pure = -1;
        if (lo0 > hi1 && lo0 > hi2) pure = 0;
        else if (lo1 > hi0 && lo1 > hi2) pure = 1;
        else if (lo2 > hi0 && lo2 > hi1) pure = 2;

        if (pure >= 0) {
            // layer by layer along the dominant axis a, with transverse axes
            // t1 = a+1, t2 = a+2 (mod 3); this thread's cell of each layer sits
            // at (lj, lk) = (tu, tv) for a = 0, (li, lk) for a = 1, (li, lj) for a = 2
            const int a = pure;
            const int h0 = a == 0 ? L::h(0, tu, tv) : (a == 1 ? L::h(tu, 0, tv) : L::h(tu, tv, 0));
            const int sa = a == 0 ? 1 : (a == 1 ? SY : SZ);
            const int s1 = a == 0 ? SY : (a == 1 ? SZ : 1);
            const int s2 = a == 0 ? SZ : (a == 1 ? 1 : SY);
            const int idx1 = a == 0 ? o0[1] + tu : (a == 1 ? o0[2] + tv : o0[0] + tu);
            const int idx2 = a == 0 ? o0[2] + tv : (a == 1 ? o0[0] + tu : o0[1] + tv);
            const int ext1 = a == 0 ? J.ext[1] : (a == 1 ? J.ext[2] : J.ext[0]);
            const int ext2 = a == 0 ? J.ext[2] : (a == 1 ? J.ext[0] : J.ext[1]);
            const int oa = a == 0 ? o0[0] : (a == 1 ? o0[1] : o0[2]);
            const int exta = a == 0 ? J.ext[0] : (a == 1 ? J.ext[1] : J.ext[2]);
            const bool col_in = idx1 >= 0 && idx2 >= 0 && idx1 < ext1 && idx2 < ext2;
            const Real c1 = Real(2 * idx1 + 1), c2 = Real(2 * idx2 + 1);
            for (int l = 0; l < T; l++) {
                const int ia = oa + l;
                if (col_in && ia >= 0 && ia < exta) {
                    const int h = h0 + l * sa;
                    const int h00 = h - sa;
                    const Real ica = Real(1) / Real(2 * ia + 1);
                    const Real g1 = c1 * ica, g2 = c2 * ica;            // weights of the t1-1 and t2-1 neighbours
                    const Real w00 = (Real(1) - g1) * (Real(1) - g2) * sW[h00];
                    const Real w01 = (Real(1) - g1) * g2 * sW[h00 - s2];
                    const Real w10 = g1 * (Real(1) - g2) * sW[h00 - s1];
                    const Real w11 = g1 * g2 * sW[h00 - s1 - s2];
                    const Col N00 = sN[h00];
                    const Real d = (w01 * ColT<Real>::sub_r(sN[h00 - s2], N00) + w10 * ColT<Real>::sub_r(sN[h00 - s1], N00) +
                                    w11 * ColT<Real>::sub_r(sN[h00 - s1 - s2], N00)) /
                                   (w00 + w01 + w10 + w11);
                    const Col Nin = ColT<Real>::add(N00, d);
                    sN[h] = ColT<Real>::add(Nin, sDI[h]);
                    sDI[h] = ColT<Real>::to_real(Nin);
                }
                __syncthreads();
            }
        } else {
            // plane by plane (li + lj + lk = m), one thread per (lj, lk) column
            const int lj = tu, lk = tv;
            for (int m = 0; m < L::NP; m++) {
                const int li = m - lj - lk;
                if (li >= 0 && li < T) {
                    const int idx[3] = {o0[0] + li, o0[1] + lj, o0[2] + lk};
                    if (idx[0] >= 0 && idx[1] >= 0 && idx[2] >= 0 && idx[0] < J.ext[0] && idx[1] < J.ext[1] &&
                        idx[2] < J.ext[2]) {
                        const int h = L::h(li, lj, lk);
                        const Col Nin = sc_entry_general<Real, T>(sN, sW, h, idx);
                        sN[h] = ColT<Real>::add(Nin, sDI[h]);
                        sDI[h] = ColT<Real>::to_real(Nin);
                    }
                }
                __syncthreads();
            }
        }

        // 4. entry columns of the tile's cells, then its downstream faces
        Real *Nout = (P.which == 1 ? G.N2 : G.N1) + (long long)J.src * G.ncell;
        for (int e = tid; e < NC; e += NT) {
            const int li = e % T, lj = (e / T) % T, lk = e / (T * T);
            const int i = o0[0] + li, j = o0[1] + lj, k = o0[2] + lk;
            if (i >= 0 && j >= 0 && k >= 0 && i < J.ext[0] && j < J.ext[1] && k < J.ext[2]) {
                const int X = J.sg[0] > 0 ? J.v[0] + i : J.v[0] - 1 - i;
                const int Y = J.sg[1] > 0 ? J.v[1] + j : J.v[1] - 1 - j;
                const int Z = J.sg[2] > 0 ? J.v[2] + k : J.v[2] - 1 - k;
                Nout[(long long)X + (long long)G.nx * ((long long)Y + (long long)G.ny * Z)] = sDI[L::h(li, lj, lk)];
            }
        }
        if (tile_self != P.skip_publish) {
            unsigned long long *const fbase = faces + tile_self * 3 * FMAX * FW::W;
            for (int q = tid; q < FaceList<T, T, T>::N; q += NT) {
                const unsigned en = __ldg(&FL.e[q]);
                const int h = remap(en & 0x3fffu);
                FW::store(fbase + (((en >> 26) & 3u) * FMAX + ((en >> 14) & 0xfffu)) * FW::W, sN[h], sW[h], epoch);
            }
        }
        __syncthreads();
    }
    // the last CTA to finish advances the epoch for the next launch
    if (tid == 0 && atomicAdd(P.done, 1u) == gridDim.x - 1) *(volatile unsigned *)P.epoch = epoch;
}

} // namespace oots
