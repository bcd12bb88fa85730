// Short-characteristics wavefront sweep (Mackey 2012, Sect. 2: column
// densities from point sources by short characteristics with the Mellema et
// al. 2006 optical-depth weighting; Sect. 5: the source sits on a cell vertex
// and each octant is traced outward independently).
//
// GB300 layout: one persistent launch covers every (grid, source, octant) of
// the call.  The octants are cut into tiles of TX x TY x TZ cells aligned to
// global multiples of the tile size (coalesced rows).  Tiles are handed out by
// an atomic ticket in order of their tile diagonal I+J+K, so every upstream
// tile was claimed by a running CTA before any tile that waits for it.
//
// Inside a tile the cells are processed plane by plane (li+lj+lk = m, one
// chain thread per (j,k) column).  The tiles are pipelined: a tile writes
// the cells of its three downstream faces to global memory as they complete,
// and a downstream tile starts each chunk of planes as soon as the face cells
// that chunk reads exist, instead of after the whole upstream tile.
//
// Hand-off without flags or fences: every published face cell is a few
// 8-byte words, each holding 4 bytes of the value and the 32-bit epoch of
// the launch (aligned 8-byte accesses are single-copy atomic).  A reader
// polls the words of the cells it needs until every one carries the current
// epoch, so each word validates itself and no progress counter, release
// fence or acquire is needed.  The epoch advances once per launch (the last
// CTA to finish stores it), so words left by earlier launches never match.
//
// Each CTA holds the chain warps, one producer warp and one writer warp.  The
// producer stages each chunk's halo cells (a compile-time list sorted by the
// first plane that reads them) from the upstream faces into shared memory,
// with bounded polling, running ahead of the chain.  The writer publishes the
// tile's downstream face cells chunk by chunk as the chain completes them, so
// the chain's plane step holds no global stores.  The chain warps form each cell's normalised neighbour
// weights off the critical path (interior cells before the first wait,
// halo-adjacent cells once their chunk's halo is staged), so a plane costs
// one weighted difference sum and one column add.  Shared-memory rows are
// padded so that a plane's cells sit in distinct banks.
#pragma once
#include "common.cuh"
#include "integrator.cuh"
#include "kernels.h"

namespace oots {

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_word(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long tagged(unsigned bits, unsigned epoch)
{
    return ((unsigned long long)epoch << 32) | bits;
}
// barrier among the chain warps only (the producer warp does not take part);
// a one-warp chain needs only the warp barrier
template <int N> __device__ __forceinline__ void chain_sync()
{
    if (N == 32) __syncwarp();
    else asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory");
}
// Chunk hand-off from the producer warp to the chain warps: named barrier
// 2 + k % 14 for chunk k, N = chain threads + 32.  The producer arrives
// (without waiting) once the chunk's halo is staged; the chain waits on it,
// blocked in hardware rather than polling.  The barrier orders the
// producer's shared-memory writes before the chain's reads.
constexpr int kHandoffBarriers = 14;
template <int N> __device__ __forceinline__ void chunk_arrive(int k)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(2 + k % kHandoffBarriers), "n"(N) : "memory");
}
template <int N> __device__ __forceinline__ void chunk_wait(int k)
{
    asm volatile("bar.sync %0, %1;" ::"r"(2 + k % kHandoffBarriers), "n"(N) : "memory");
}

// A published face cell (column N_out and weight factor W) as tagged words:
// mixed path {N.hi}, {N.lo}, {W}; FP64 path both halves of N and of W.
template <typename Real> struct FaceWords;
template <> struct FaceWords<float> {
    enum { W = 3 };
    static __device__ __forceinline__ void store(unsigned long long *p, ff N, float w, unsigned e)
    {
        st_word(p + 0, tagged(__float_as_uint(N.hi), e));
        st_word(p + 1, tagged(__float_as_uint(N.lo), e));
        st_word(p + 2, tagged(__float_as_uint(w), e));
    }
    // true once every word carries epoch e
    static __device__ __forceinline__ bool load(const unsigned long long *p, unsigned e, ff &N, float &w)
    {
        const unsigned long long a = ld_word(p + 0), b = ld_word(p + 1), c = ld_word(p + 2);
        N = ff{__uint_as_float((unsigned)a), __uint_as_float((unsigned)b)};
        w = __uint_as_float((unsigned)c);
        return (unsigned)(a >> 32) == e && (unsigned)(b >> 32) == e && (unsigned)(c >> 32) == e;
    }
};
template <> struct FaceWords<double> {
    enum { W = 4 };
    static __device__ __forceinline__ void store(unsigned long long *p, double N, double w, unsigned e)
    {
        const unsigned long long n = (unsigned long long)__double_as_longlong(N), v = (unsigned long long)__double_as_longlong(w);
        st_word(p + 0, tagged((unsigned)n, e));
        st_word(p + 1, tagged((unsigned)(n >> 32), e));
        st_word(p + 2, tagged((unsigned)v, e));
        st_word(p + 3, tagged((unsigned)(v >> 32), e));
    }
    static __device__ __forceinline__ bool load(const unsigned long long *p, unsigned e, double &N, double &w)
    {
        const unsigned long long a = ld_word(p + 0), b = ld_word(p + 1), c = ld_word(p + 2), d = ld_word(p + 3);
        N = __longlong_as_double((long long)(((b & 0xffffffffull) << 32) | (a & 0xffffffffull)));
        w = __longlong_as_double((long long)(((d & 0xffffffffull) << 32) | (c & 0xffffffffull)));
        return (unsigned)(a >> 32) == e && (unsigned)(b >> 32) == e && (unsigned)(c >> 32) == e &&
               (unsigned)(d >> 32) == e;
    }
};

// Shared-memory layout of a sweep tile: a one-cell halo on the three upstream
// sides, with the row strides padded so that the cells of one plane
// li+lj+lk = m handled by a warp (lane t: lj = t % TY, lk = t / TY) fall in
// distinct banks for 4-byte arrays and in distinct bank pairs within each
// half-warp for 8-byte arrays.  Along a plane the address moves by SY - 1 per
// lj and by SZ - 1 per lk.
constexpr bool plane_conflict_free(int a, int b, int TY, int NT)
{
    for (int w = 0; w < NT / 32; w++) {
        bool b32[32] = {}, b16[2][16] = {};
        for (int l = 0; l < 32; l++) {
            const int t = 32 * w + l, lj = t % TY, lk = t / TY;
            const int off = lj * a + lk * b;
            if (b32[off % 32]) return false;
            b32[off % 32] = true;
            if (b16[l / 16][off % 16]) return false;
            b16[l / 16][off % 16] = true;
        }
    }
    return true;
}
constexpr int pick_plane_stride(int SY, int HY, int TY, int NT)
{
    for (int s = SY * HY; s < SY * HY + 64; s++)
        if (plane_conflict_free(SY - 1, s - 1, TY, NT)) return s;
    return SY * HY;
}

template <int TX, int TY, int TZ> struct TileLayout {
    static constexpr int HX = TX + 1, HY = TY + 1, HZ = TZ + 1;
    static constexpr int NT = TY * TZ;
    static constexpr int SY = (HX % 2 == 0) ? HX : HX + 1;          // SY - 1 odd
    static constexpr int SZ = pick_plane_stride(SY, HY, TY, NT);
    static constexpr int HSZ = HZ * SZ;                               // entries per array
    static constexpr int NP = TX + TY + TZ - 2;                       // planes of a tile
    static constexpr int NE = HY * HZ + TX * HZ + TX * TY;            // halo cells
    static constexpr int FMAX = (TY * TZ > TX * TZ ? (TY * TZ > TX * TY ? TY * TZ : TX * TY)
                                                   : (TX * TZ > TX * TY ? TX * TZ : TX * TY));
    static constexpr OOTS_HD int h(int li, int lj, int lk) { return (lk + 1) * SZ + (lj + 1) * SY + (li + 1); }
    static_assert(HSZ < (1 << 14) && FMAX <= (1 << 12), "halo entry packing");
};

// The halo cells of a tile sorted by the first plane that reads them (its
// key): an X-face cell (-1, lj, lk) is first read by plane max(lj,0) +
// max(lk,0), a Y-face cell (li, -1, lk) by li + max(lk,0), a Z-face cell
// (li, lj, -1) by li + lj.  Each entry packs the halo index (14 bits), the
// index within the upstream face (12 bits), the face (2 bits) and the mask of
// tile steps (-x, -y, -z) from this tile to the tile that published it.
template <int TX, int TY, int TZ> struct HaloList {
    unsigned e[TileLayout<TX, TY, TZ>::NE];
    unsigned short start[TileLayout<TX, TY, TZ>::NP + 1];
};
template <int TX, int TY, int TZ>
constexpr void halo_entry(int q, int &key, unsigned &packed)
{
    typedef TileLayout<TX, TY, TZ> L;
    int li = 0, lj = 0, lk = 0, face = 0, mask = 0, fq = 0;
    if (q < L::HY * L::HZ) {
        lj = q % L::HY - 1; lk = q / L::HY - 1; li = -1; face = 0;
        key = (lj > 0 ? lj : 0) + (lk > 0 ? lk : 0);
        mask = 1 | (lj < 0 ? 2 : 0) | (lk < 0 ? 4 : 0);
        fq = (lk < 0 ? TZ - 1 : lk) * TY + (lj < 0 ? TY - 1 : lj);
    } else if (q < L::HY * L::HZ + TX * L::HZ) {
        const int r = q - L::HY * L::HZ;
        li = r % TX; lk = r / TX - 1; lj = -1; face = 1;
        key = li + (lk > 0 ? lk : 0);
        mask = 2 | (lk < 0 ? 4 : 0);
        fq = (lk < 0 ? TZ - 1 : lk) * TX + li;
    } else {
        const int r = q - L::HY * L::HZ - TX * L::HZ;
        li = r % TX; lj = r / TX; lk = -1; face = 2;
        key = li + lj;
        mask = 4;
        fq = lj * TX + li;
    }
    packed = (unsigned)L::h(li, lj, lk) | ((unsigned)fq << 14) | ((unsigned)face << 26) | ((unsigned)mask << 28);
}
template <int TX, int TY, int TZ>
constexpr HaloList<TX, TY, TZ> make_halo_list()
{
    typedef TileLayout<TX, TY, TZ> L;
    HaloList<TX, TY, TZ> H{};
    int cnt[L::NP + 1] = {};
    for (int q = 0; q < L::NE; q++) {
        int key = 0; unsigned p = 0;
        halo_entry<TX, TY, TZ>(q, key, p);
        cnt[key + 1]++;
    }
    for (int k = 0; k < L::NP; k++) cnt[k + 1] += cnt[k];
    for (int k = 0; k <= L::NP; k++) H.start[k] = (unsigned short)cnt[k];
    for (int q = 0; q < L::NE; q++) {
        int key = 0; unsigned p = 0;
        halo_entry<TX, TY, TZ>(q, key, p);
        H.e[cnt[key]++] = p;
    }
    return H;
}
template <int TX, int TY, int TZ>
__device__ const HaloList<TX, TY, TZ> g_halo_list = make_halo_list<TX, TY, TZ>();

// The tile's own downstream face cells (li = TX-1, lj = TY-1, lk = TZ-1) sorted
// by the plane that completes them, packed like the halo list (halo index,
// index within the face, face); a cell on two or three faces appears once per
// face.  The writer warp publishes them chunk by chunk.
template <int TX, int TY, int TZ> struct FaceList {
    enum { N = TY * TZ + TX * TZ + TX * TY };
    unsigned e[N];
    unsigned short start[TileLayout<TX, TY, TZ>::NP + 1];
};
template <int TX, int TY, int TZ>
constexpr void face_entry(int q, int &key, unsigned &packed)
{
    typedef TileLayout<TX, TY, TZ> L;
    int li = 0, lj = 0, lk = 0, face = 0, fq = 0;
    if (q < TY * TZ) {
        lj = q % TY; lk = q / TY; li = TX - 1; face = 0; fq = lk * TY + lj;
    } else if (q < TY * TZ + TX * TZ) {
        const int r = q - TY * TZ;
        li = r % TX; lk = r / TX; lj = TY - 1; face = 1; fq = lk * TX + li;
    } else {
        const int r = q - TY * TZ - TX * TZ;
        li = r % TX; lj = r / TX; lk = TZ - 1; face = 2; fq = lj * TX + li;
    }
    key = li + lj + lk;
    packed = (unsigned)L::h(li, lj, lk) | ((unsigned)fq << 14) | ((unsigned)face << 26);
}
template <int TX, int TY, int TZ>
constexpr FaceList<TX, TY, TZ> make_face_list()
{
    typedef TileLayout<TX, TY, TZ> L;
    typedef FaceList<TX, TY, TZ> FL;
    FL F{};
    int cnt[L::NP + 1] = {};
    for (int q = 0; q < FL::N; q++) {
        int key = 0; unsigned p = 0;
        face_entry<TX, TY, TZ>(q, key, p);
        cnt[key + 1]++;
    }
    for (int k = 0; k < L::NP; k++) cnt[k + 1] += cnt[k];
    for (int k = 0; k <= L::NP; k++) F.start[k] = (unsigned short)cnt[k];
    for (int q = 0; q < FL::N; q++) {
        int key = 0; unsigned p = 0;
        face_entry<TX, TY, TZ>(q, key, p);
        F.e[cnt[key]++] = p;
    }
    return F;
}
template <int TX, int TY, int TZ>
__device__ const FaceList<TX, TY, TZ> g_face_list = make_face_list<TX, TY, TZ>();

// Whether some grid of the launch has not reached its end time (true when
// the launch does not say how many grids it holds).  A launch whose grids are
// all done claims no tile, so substeps past the end cost little.
template <typename Real> __device__ __forceinline__ bool sweep_live(const SweepParams<Real> &P)
{
    if (P.ngrid <= 0) return true;
    for (int q = 0; q < P.ngrid; q++)
        if (!P.grids[q].st->done) return true;
    return false;
}

template <typename Real, int TX, int TY, int TZ, int MODE>
__global__ void __launch_bounds__(TY *TZ + 64)
sweep_kernel(SweepParams<Real> P)
{
    typedef typename ColT<Real>::type Col;
    typedef TileLayout<TX, TY, TZ> L;
    constexpr int NT = L::NT;                    // chain threads
    constexpr int NC = TX * TY * TZ;
    constexpr int NP = L::NP;
    constexpr int FMAX = L::FMAX;
    constexpr int HSZ = L::HSZ;
    constexpr int SY = L::SY, SZ = L::SZ;
    static_assert(NT % 32 == 0, "the chain threads fill whole warps");
    static_assert(NC % (4 * NT) == 0, "pre-pass batches of four cells per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // every array is indexed by the padded halo index L::h(li, lj, lk)
    Col *sN = reinterpret_cast<Col *>(smem_raw);       // N_out of the cell
    Real *sW = reinterpret_cast<Real *>(sN + HSZ);     // 1/max(dtau, tau0); 0 outside the octant
    Real *sDI = sW + HSZ;                              // increment n x ds (MODE 1: x0), then N_in
    Real *sQ = sDI + HSZ;                              // 3 x HSZ neighbour weights (see below)
    unsigned char *sMode = reinterpret_cast<unsigned char *>(sQ + 3 * HSZ); // chain mode (see below)
    __shared__ unsigned s_ticket;
    __shared__ volatile int s_done;              // chunks the chain has completed (for the writer)
    __shared__ double s_bud[3];
    const HaloList<TX, TY, TZ> &HL = g_halo_list<TX, TY, TZ>;
    const FaceList<TX, TY, TZ> &FL = g_face_list<TX, TY, TZ>;

    typedef FaceWords<Real> FW;
    unsigned long long *const faces = P.faces;
    // the epoch of this launch: one past the last finished launch's (read
    // before this CTA reports done, so before the last CTA advances it)
    const unsigned epoch = *(volatile unsigned *)P.epoch + 1u;
    const int tid = threadIdx.x;
    const int clj = tid % TY, clk = tid / TY;    // chain threads: own (j,k) column
    // planes per chunk; at most kHandoffBarriers chunks per tile, so no
    // hand-off barrier is reused within a tile
    const int chunk = max(P.chunk > 0 ? P.chunk : 4, (NP + kHandoffBarriers - 1) / kHandoffBarriers);
    double bud_ions = 0.0, bud_rec = 0.0;
    int bud_grid = -1;

    // halo-index strides of the dominant axis a and of its two transverse axes
    auto str_a = [](int a) { return a == 0 ? 1 : (a == 1 ? SY : SZ); };
    auto str_t1 = [](int a) { return a == 0 ? SY : (a == 1 ? SZ : 1); };
    auto str_t2 = [](int a) { return a == 0 ? SZ : (a == 1 ? 1 : SY); };

    // Normalised weights of the (t1-1), (t2-1) and (t1-1,t2-1) upwind
    // neighbours relative to the (0,0) one, from the 1-D weights g1, g2 held
    // in sQ[h], sQ[HSZ+h] and the neighbours' optical-depth factors:
    // N_in = N00 + q01 (N01 - N00) + q10 (N10 - N00) + q11 (N11 - N00).
    auto weights = [&](int h, unsigned mode) {
        const int a = mode & 3;
        const int h00 = h - str_a(a), s1 = str_t1(a), s2 = str_t2(a);
        const Real g1 = sQ[h], g2 = sQ[HSZ + h];
        const Real w00 = (Real(1) - g1) * (Real(1) - g2) * sW[h00];
        const Real w01 = (mode & 8) ? (Real(1) - g1) * g2 * sW[h00 - s2] : Real(0);
        const Real w10 = (mode & 4) ? g1 * (Real(1) - g2) * sW[h00 - s1] : Real(0);
        const Real w11 = ((mode & 12) == 12) ? g1 * g2 * sW[h00 - s1 - s2] : Real(0);
        const Real r = Real(1) / (w00 + w01 + w10 + w11);
        sQ[h] = w01 * r;
        sQ[HSZ + h] = w10 * r;
        sQ[2 * HSZ + h] = w11 * r;
    };
    // a regular cell one of whose upwind neighbours lies in the halo
    auto on_halo = [](int li, int lj, int lk, unsigned mode) {
        const int a = mode & 3;
        const int la = a == 0 ? li : (a == 1 ? lj : lk);
        const int l1 = a == 0 ? lj : (a == 1 ? lk : li);
        const int l2 = a == 0 ? lk : (a == 1 ? li : lj);
        return la == 0 || ((mode & 4) && l1 == 0) || ((mode & 8) && l2 == 0);
    };

    const bool live = tid == 0 && sweep_live(P);     // read by thread 0 only
    for (;;) {
        if (tid == 0) {
            unsigned t = live ? atomicAdd(P.ticket, 1u) : (unsigned)P.nitems;
            // a grid that has reached its end time skips every tile (all its
            // tiles skip, so no wait is left pending)
            if (t < (unsigned)P.nitems && P.grids[P.jobs[P.items[t].job].grid].st->done) t |= 0x80000000u;
            s_ticket = t;
            s_done = 0;
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

        if (tid >= NT + 32) {
            // ---------------- writer warp ----------------
            // after chunk k, the face cells its planes completed go out as tagged
            // words (the chain's barrier and the shared counter order the chain's
            // shared-memory writes before these reads)
            const int lane = tid - NT - 32;
            if (tile_self != P.skip_publish) {
                unsigned long long *const fbase = faces + tile_self * 3 * FMAX * FW::W;
                int k = 0;
                for (int m0 = 0; m0 < NP; m0 += chunk, k++) {
                    const int m1 = min(m0 + chunk, NP);
                    long long spins = 0;
                    while (s_done <= k) {
                        if (++spins > (P.spin_limit << 4)) { atomicCAS(P.err, 0, (int)DEVERR_TIMEOUT); break; }
                        __nanosleep(32);
                    }
                    __threadfence_block();
                    for (int q = FL.start[m0] + lane; q < FL.start[m1]; q += 32) {
                        const unsigned en = __ldg(&FL.e[q]);
                        const int h = en & 0x3fffu;
                        FW::store(fbase + (((en >> 26) & 3u) * FMAX + ((en >> 14) & 0xfffu)) * FW::W, sN[h], sW[h], epoch);
                    }
                }
            }
        } else if (tid >= NT) {
            // ---------------- producer warp ----------------
            const int lane = tid - NT;
            // zero the halo (read as absent until staged)
            for (int q = lane; q < L::NE; q += 32) {
                const int h = __ldg(&HL.e[q]) & 0x3fffu;
                sN[h] = ColT<Real>::zero();
                sW[h] = Real(0);
            }
            __syncwarp();
            const long long sx = 1, sy = J.nt[0], sz = (long long)J.nt[0] * J.nt[1];
            const unsigned have = (it.I > 0 ? 1u : 0u) | (it.J > 0 ? 2u : 0u) | (it.K > 0 ? 4u : 0u);
            int k = 0;
            for (int m0 = 0; m0 < NP; m0 += chunk, k++) {
                const int m1 = min(m0 + chunk, NP);
                // stage the halo cells first read by planes [m0, m1), four per lane
                // in flight, polling each until all its words carry this epoch
                const int b1 = HL.start[m1];
                for (int base = HL.start[m0] + lane; base < b1; base += 128) {
                    unsigned en[4];
                    long long o[4];
                    bool ok[4];
                    Col vN[4];
                    Real vW[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int q = base + 32 * u;
                        en[u] = q < b1 ? __ldg(&HL.e[q]) : 0u;
                        const unsigned mask = en[u] >> 28;
                        ok[u] = true;
                        o[u] = 0;
                        if (q < b1 && (mask & ~have) == 0) {
                            const long long src = tile_self - ((mask & 1) ? sx : 0) - ((mask & 2) ? sy : 0) - ((mask & 4) ? sz : 0);
                            o[u] = ((src * 3 + (long long)((en[u] >> 26) & 3u)) * FMAX + ((en[u] >> 14) & 0xfffu)) * FW::W;
                            ok[u] = FW::load(faces + o[u], epoch, vN[u], vW[u]);
                        } else {
                            en[u] = 0u;           // no upstream tile: the cell stays absent
                        }
                    }
                    long long spins = 0;
                    unsigned ns = 32;
                    while (!(ok[0] && ok[1] && ok[2] && ok[3])) {
                        if (++spins > P.spin_limit) { atomicCAS(P.err, 0, (int)DEVERR_TIMEOUT); break; }
                        if ((spins & 31) == 0 && *(volatile int *)P.err != 0) break;   // another tile gave up
                        __nanosleep(ns);
                        if (ns < 256) ns <<= 1;
#pragma unroll
                        for (int u = 0; u < 4; u++)
                            if (!ok[u]) ok[u] = FW::load(faces + o[u], epoch, vN[u], vW[u]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (en[u]) {
                            sN[en[u] & 0x3fffu] = ok[u] ? vN[u] : ColT<Real>::zero();
                            sW[en[u] & 0x3fffu] = ok[u] ? vW[u] : Real(0);
                        }
                }
                __syncwarp();
                chunk_arrive<NT + 32>(k);
            }
        } else {
            // ---------------- chain warps ----------------
            // 1. own cells: increments, weight factors, chain modes (loads in
            //    batches of four cells per thread)
            for (int e0 = tid; e0 < NC; e0 += 4 * NT) {
                long long gq[4];
                bool in[4];
                Real nv[4], xv[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int e = e0 + u * NT;
                    const int li = e % TX, lj = (e / TX) % TY, lk = e / (TX * TY);
                    const int i = i0 + li, j = j0 + lj, k = k0 + lk;
                    in[u] = i >= 0 && j >= 0 && k >= 0 && i < J.ext[0] && j < J.ext[1] && k < J.ext[2];
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
                    const int li = e % TX, lj = (e / TX) % TY, lk = e / (TX * TY);
                    const int i = i0 + li, j = j0 + lj, k = k0 + lk;
                    const int h = L::h(li, lj, lk);
                    Real dN = Real(0), wf = Real(0);
                    // chain mode: bits 0-1 dominant axis; bit 2 / bit 3: the t1-1 / t2-1
                    // neighbour exists (inside the octant); bit 4 the vertex cell; bit 5
                    // tied dominant axis (general path); bit 7 outside the octant
                    unsigned char mode = 0x80;
                    if (in[u]) {
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
                            sQ[h] = Real(c2i[t1]) / Real(c2i[a]);
                            sQ[HSZ + h] = Real(c2i[t2]) / Real(c2i[a]);
                        }
                        const Real c0 = Real(i) + Real(0.5), c1 = Real(j) + Real(0.5), c2 = Real(k) + Real(0.5);
                        const Real cm = m_max(c0, m_max(c1, c2));
                        const Real ds = dx * m_sqrt(c0 * c0 + c1 * c1 + c2 * c2) / cm;
                        if (MODE == 0) {
                            dN = nv[u] * xv[u] * ds;
                            wf = Real(1) / m_max(sig * dN, tau0);
                        } else {
                            dN = xv[u];                            // A1: x0, integrated in the chain
                            wf = Real(1);                          // set in the chain
                        }
                    }
                    sN[h] = ColT<Real>::zero();
                    sW[h] = wf;
                    sDI[h] = dN;
                    sMode[h] = mode;
                }
            }
            chain_sync<NT>();
            // interior cells: neighbour weights before the first wait
            if (MODE == 0) {
                for (int li = 0; li < TX; li++) {
                    const int h = L::h(li, clj, clk);
                    const unsigned mode = sMode[h];
                    if (!(mode & 0xB0) && !on_halo(li, clj, clk, mode)) weights(h, mode);
                }
            }


            int k = 0;
            for (int m0 = 0; m0 < NP; m0 += chunk, k++) {
                const int m1 = min(m0 + chunk, NP);
                // the chunk's halo is staged (the producer's upstream waits are
                // bounded, so it always arrives)
                chunk_wait<NT + 32>(k);
                // halo-adjacent cells of this chunk: neighbour weights
                if (MODE == 0) {
                    for (int m = m0; m < m1; m++) {
                        const int li = m - clj - clk;
                        if (li < 0 || li >= TX) continue;
                        const int h = L::h(li, clj, clk);
                        const unsigned mode = sMode[h];
                        if (!(mode & 0xB0) && on_halo(li, clj, clk, mode)) weights(h, mode);
                    }
                }
                // 2. plane-by-plane recurrence
                for (int m = m0; m < m1; m++) {
                    const int li = m - clj - clk;
                    if (li >= 0 && li < TX) {
                        const int lj = clj, lk = clk;
                        const int i = i0 + li, j = j0 + lj, k = k0 + lk;
                        const int h = L::h(li, lj, lk);
                        const unsigned mode = sMode[h];
                        Col Nout = ColT<Real>::zero();
                        Real wout = Real(0);
                        if (!(mode & 0x80)) {
                            wout = sW[h];
                            const Real dval = sDI[h];
                            if (MODE == 0 && !(mode & 0x30)) {
                                // one dominant axis: weighted differences to the (0,0) neighbour
                                const int a = mode & 3;
                                const int h00 = h - str_a(a), s1 = str_t1(a), s2 = str_t2(a);
                                const int h01 = (mode & 8) ? h00 - s2 : h00;
                                const int h10 = (mode & 4) ? h00 - s1 : h00;
                                const int h11 = ((mode & 12) == 12) ? h00 - s1 - s2 : h00;
                                const Col N00 = sN[h00];
                                const Real d = sQ[h] * ColT<Real>::sub_r(sN[h01], N00)
                                             + sQ[HSZ + h] * ColT<Real>::sub_r(sN[h10], N00)
                                             + sQ[2 * HSZ + h] * ColT<Real>::sub_r(sN[h11], N00);
                                Nout = ColT<Real>::add(N00, d + dval);
                                sDI[h] = ColT<Real>::to_real(ColT<Real>::add(N00, d));
                            } else if (MODE == 0 && (mode & 0x20)) {
                                // tied dominant axes: the average over the tied axes of
                                // each axis's normalised interpolation, as weighted
                                // differences to the neighbour one step back along every
                                // tied axis (it always carries weight; the weights of all
                                // terms sum to one)
                                const int idx[3] = {i, j, k};
                                const int c2[3] = {2 * i + 1, 2 * j + 1, 2 * k + 1};
                                const int cm = max(c2[0], max(c2[1], c2[2]));
                                const Col Nref = sN[h - (c2[0] == cm ? str_a(0) : 0) - (c2[1] == cm ? str_a(1) : 0) -
                                                    (c2[2] == cm ? str_a(2) : 0)];
                                const Real inv_nt = Real(1) / Real((c2[0] == cm) + (c2[1] == cm) + (c2[2] == cm));
                                Real d = Real(0);
#pragma unroll
                                for (int a = 0; a < 3; a++) {
                                    if (c2[a] != cm) continue;
                                    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
                                    const int ha = h - str_a(a), s1 = str_t1(a), s2 = str_t2(a);
                                    const Real w1 = Real(c2[t1]) / Real(c2[a]);   // weight of the t1-1 neighbour
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
                                    if (ws > Real(0)) {
                                        const Real r = inv_nt / ws;
                                        d += r * (wv[0] * dv[0] + wv[1] * dv[1] + wv[2] * dv[2] + wv[3] * dv[3]);
                                    }
                                }
                                Nout = ColT<Real>::add(Nref, d + dval);
                                sDI[h] = ColT<Real>::to_real(ColT<Real>::add(Nref, d));
                            } else {
                                Col Nin = ColT<Real>::zero();
                                if (!(mode & 0x30)) {
                                    // (MODE 1) one dominant axis: bilinear weights times the
                                    // neighbours' factors, normalised once
                                    const int a = mode & 3;
                                    const int h00 = h - str_a(a), s1 = str_t1(a), s2 = str_t2(a);
                                    const Real g1 = sQ[h], g2 = sQ[HSZ + h];
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
                                    // tied dominant axes: average of the interpolations along each
                                    const int idx[3] = {i, j, k};
                                    const int loc[3] = {li, lj, lk};
                                    const int c2[3] = {2 * i + 1, 2 * j + 1, 2 * k + 1};
                                    const int cm = max(c2[0], max(c2[1], c2[2]));
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
                                                const int hn = L::h(nb[0], nb[1], nb[2]);
                                                const Real wg = (e1 ? w1 : Real(1) - w1) * (e2 ? w2 : Real(1) - w2);
                                                const Real w = wg * sW[hn];
                                                acc = ColT<Real>::fma_w(acc, w, sN[hn]);
                                                ws += w;
                                            }
                                        }
                                        if (ws > Real(0)) sum = ColT<Real>::addc(sum, ColT<Real>::div(acc, ws));
                                    }
                                    Nin = ColT<Real>::div(sum, Real(ntied));
                                }
                                const Real nin_r = ColT<Real>::to_real(Nin);
                                sDI[h] = nin_r;
                                if (MODE == 0) {
                                    Nout = ColT<Real>::add(Nin, dval);
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
                                    IntResult<Real> R = integrate_cell<Real, 1>(C, dval, dt, sig);
                                    Real dtau_eff = -R.lnfav;
                                    if (!(dtau_eff >= Real(0))) dtau_eff = Real(0);
                                    Nout = ColT<Real>::add(Nin, dtau_eff / sig);
                                    wout = Real(1) / m_max(dtau_eff, tau0);
                                    sW[h] = wout;
                                    if (dt > Real(0)) {
                                        G.xout[g] = R.x;
                                        const double nV = double(n) * G.st->cell_volume;
                                        bud_ions += nV * double(dval - R.x);
                                        bud_rec += nV * double(R.IR);
                                        bud_grid = J.grid;
                                    }
                                }
                            }
                            sN[h] = Nout;
                        }
                    }
                    chain_sync<NT>();
                }
                // 3. chunk done: its face cells go to the writer warp
                if (tid == 0) { __threadfence_block(); s_done = k + 1; }
            }

            // 4. entry columns of the tile's cells
            Real *Nout = (P.which == 1 ? G.N2 : G.N1) + (long long)J.src * G.ncell;
            for (int e = tid; e < NC; e += NT) {
                const int li = e % TX, lj = (e / TX) % TY, lk = e / (TX * TY);
                const int i = i0 + li, j = j0 + lj, k = k0 + lk;
                if (i >= 0 && j >= 0 && k >= 0 && i < J.ext[0] && j < J.ext[1] && k < J.ext[2]) {
                    const int X = J.sg[0] > 0 ? J.v[0] + i : J.v[0] - 1 - i;
                    const int Y = J.sg[1] > 0 ? J.v[1] + j : J.v[1] - 1 - j;
                    const int Z = J.sg[2] > 0 ? J.v[2] + k : J.v[2] - 1 - k;
                    const long long g = (long long)X + (long long)G.nx * ((long long)Y + (long long)G.ny * Z);
                    Nout[g] = sDI[L::h(li, lj, lk)];
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
    // the last CTA to finish advances the epoch for the next launch
    if (tid == 0 && atomicAdd(P.done, 1u) == gridDim.x - 1) *(volatile unsigned *)P.epoch = epoch;
}

} // namespace oots

#include "sweep_tp.cuh"

namespace oots {

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
template <typename Real, int TX, int TY, int TZ>
constexpr size_t sweep_smem()
{
    return (size_t)TileLayout<TX, TY, TZ>::HSZ * (sizeof(typename ColT<Real>::type) + 5 * sizeof(Real) + 1);
}

template <typename Real, int TX, int TY, int TZ, int MODE>
static cudaError_t launch_shape(const SweepParams<Real> &P, int nblocks, cudaStream_t s)
{
    constexpr size_t sm = sweep_smem<Real, TX, TY, TZ>();
    sweep_kernel<Real, TX, TY, TZ, MODE><<<nblocks, TY * TZ + 64, sm, s>>>(P);
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
    if (shape == SHAPE_TP8) return (int)sweep_tp_smem<Real, 8>() <= max_optin_smem() && sweep_shape_ok<Real>(4);
    if (shape == SHAPE_TP16) return (int)sweep_tp_smem<Real, 16>() <= max_optin_smem() && sweep_shape_ok<Real>(0);
    size_t sm = 0;
#define OOTS_SM(ID, TX, TY, TZ) if (shape == ID) sm = sweep_smem<Real, TX, TY, TZ>();
    OOTS_SHAPES(OOTS_SM)
#undef OOTS_SM
    return sm > 0 && (int)sm <= max_optin_smem();
}

template <typename Real>
int sweep_occupancy(int shape, int mode)
{
    int nb = 0;
    cudaError_t e = cudaSuccess;
    if (is_tp_shape(shape)) {
        if (mode == 1) return sweep_occupancy<Real>(tp_twin(shape), 1);
        if (shape == SHAPE_TP8)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_tp_kernel<Real, 8>, 64, sweep_tp_smem<Real, 8>());
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_tp_kernel<Real, 16>, 64, sweep_tp_smem<Real, 16>());
        return (e == cudaSuccess && nb > 0) ? nb : 1;
    }
#define OOTS_OCC(ID, TX, TY, TZ)                                                                      \
    if (shape == ID) {                                                                                \
        constexpr size_t sm = sweep_smem<Real, TX, TY, TZ>();                                         \
        if (mode == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<Real, TX, TY, TZ, 0>, TY * TZ + 64, sm); \
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<Real, TX, TY, TZ, 1>, TY * TZ + 64, sm); \
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
    if (is_tp_shape(shape)) {
        if (mode == 1) return launch_sweep<Real>(P, tp_twin(shape), 1, nblocks, s);
        if (shape == SHAPE_TP8) sweep_tp_kernel<Real, 8><<<(int)nb, 64, sweep_tp_smem<Real, 8>(), s>>>(P);
        else sweep_tp_kernel<Real, 16><<<(int)nb, 64, sweep_tp_smem<Real, 16>(), s>>>(P);
        return cudaGetLastError();
    }
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
cudaError_t launch_pack_nx(const GridDev<Real> *grids, int ngrid, int which, int shape, long long max_elems, int nsm,
                           cudaStream_t s)
{
    if (ngrid <= 0 || max_elems <= 0) return cudaSuccess;
    if (ngrid > 65535) return cudaErrorInvalidValue;
    long long nb = (max_elems + 255) / 256;
    const long long cap = (long long)(nsm > 0 ? nsm : 1) * 8;       // 2048 threads per SM
    if (nb > cap) nb = cap;
    const dim3 grid((unsigned)nb, (unsigned)ngrid);
    if (shape == SHAPE_TP16) pack_nx_kernel<Real, 16><<<grid, 256, 0, s>>>(grids, which);
    else pack_nx_kernel<Real, 8><<<grid, 256, 0, s>>>(grids, which);
    return cudaGetLastError();
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
    if ((int)sweep_tp_smem<Real, 8>() <= max_optin_smem()) {
        e2 = cudaFuncSetAttribute(sweep_tp_kernel<Real, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sweep_tp_smem<Real, 8>());
        if (e2 != cudaSuccess) e = e2;
    }
    if ((int)sweep_tp_smem<Real, 16>() <= max_optin_smem()) {
        e2 = cudaFuncSetAttribute(sweep_tp_kernel<Real, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sweep_tp_smem<Real, 16>());
        if (e2 != cudaSuccess) e = e2;
    }
    return e;
}


} // namespace oots
