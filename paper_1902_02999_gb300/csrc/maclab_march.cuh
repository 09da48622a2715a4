// maclab_march.cuh -- the row-marching step kernel of MacLABSWE (Zhou,
// arXiv:1902.02999, Section 3, Eqs. Mac.lb.6 / Mac.lb.7 in the perturbation
// form of maclab_kernels.cuh) for sm_103a.
//
// A warp owns a strip of 64 grid columns and a block of rows (a "strip
// block") and walks down the rows.  Lane k derives the node pair at columns
// X0 + 2k, X0 + 2k + 1 of each row: the source quantities of Section 3 (the
// eight outgoing equilibrium differences with the source halves of the bed
// and force terms, derive2), written to a three-row ring in the warp's
// shared memory (o1, o2, o4, o5 and (eta, D) split by column parity, so
// that a warp reading one column per lane has no bank conflicts).  When
// row r is derived, output row r - 1 is complete: each lane updates its two
// nodes (x, x + 1) from the ring (rows r - 2, r - 1), its own registers
// (row r, o3 and its own (eta, D) of the two rows above) and two warp
// shuffles (o8, o6 of row r from the neighbouring lanes).  The update runs
// the streamed sums and the final arithmetic of the tile kernel with one
// node per lane of the paired FP32 instructions; every lane takes the same
// operations in the same order, so the states are bitwise those of the tile
// kernel.  A strip writes columns X0 + 2 .. X0 + 61 (OUT = 60: lanes 0 and
// 31 only supply the neighbours) and rows j0 .. j1 - 1; rows j0 - 1 and j1
// are derived only.
//
// Raw rows are staged two rows ahead by cp.async into lane-private slots of
// the warp's shared memory, so no row waits for memory after the first two
// and no prefetch occupies registers; raw and derived rows share the ring
// period 3, and the row loop is unrolled three times with compile-time
// slots.  Strip blocks whose rows and columns lie inside the grid and whose
// written nodes are all fluid or Dirichlet nodes without a bounce-back link
// ("plain" interior blocks, flagged by the host) take a path with no node
// types at all; the others resolve rows and columns through the edge rules.
// The host orders the strip blocks tall first and short last (blocks start
// in index order as warp slots free up), so the last wave is short.
//
// After its rows, a warp updates the nodes of its strip block that have a
// bounce-back link (general_node, old state only) and then, when every
// Dirichlet node's inward node lies in the same strip block, the block's
// Dirichlet nodes from the new values its own lanes wrote (__syncwarp
// orders those writes before the reads).
#pragma once
#include "maclab_kernels.cuh"

namespace maclab {
namespace march {

constexpr int WARPS = 4;             // warps (strip blocks) per block
constexpr int THREADS = 32 * WARPS;
#ifndef MACLAB_MARCH_OUT
#define MACLAB_MARCH_OUT 60
#endif
constexpr int OUT = MACLAB_MARCH_OUT;  // columns written per strip: 62 or 60
constexpr int HALF = (62 - OUT) / 2;   // derived columns beyond the one-column halo, per side
constexpr int MIN_ROWS = 8;          // rows per strip block, at least
#ifndef MACLAB_MARCH_WAVES
#define MACLAB_MARCH_WAVES 6
#endif
constexpr int WAVES = MACLAB_MARCH_WAVES;  // uniform split: strip blocks per resident warp slot
// guided split (GUIDED_PHI > 0): one wave of tall strip blocks covering the
// fraction GUIDED_PHI of the rows, then blocks GUIDED_DIV times shorter
#ifndef MACLAB_MARCH_GUIDED_PHI
#define MACLAB_MARCH_GUIDED_PHI 0.6
#endif
#ifndef MACLAB_MARCH_GUIDED_DIV
#define MACLAB_MARCH_GUIDED_DIV 6
#endif

// Strip s derives the 64 columns from X0 = OUT s - 2 and writes local
// columns 1 + HALF .. 62 - HALF: with OUT = 62 global columns 62 s - 1 ..
// 62 s + 60, with OUT = 60 columns 60 s .. 60 s + 59.
__host__ __device__ constexpr int first_col(int s) { return OUT * s - 2; }
// strip of the node at column x (the strip that writes it)
__host__ __device__ constexpr int strip_of(int x) { return (x + 1 - HALF) / OUT; }
__host__ __device__ constexpr int strips(int nx) { return strip_of(nx - 1) + 1; }

constexpr int AHEAD = 2;  // rows of loads in flight per warp
#ifndef MACLAB_MARCH_CARRY
#define MACLAB_MARCH_CARRY 2
#endif
constexpr int CARRY = MACLAB_MARCH_CARRY;  // 1: o3 in registers; 2: also the lane's own (eta, D)

#ifndef MACLAB_MARCH_MINB_F32
#define MACLAB_MARCH_MINB_F32 5
#endif
template <typename T> struct MinBlocks { static constexpr int value = MACLAB_MARCH_MINB_F32; };
template <> struct MinBlocks<double> { static constexpr int value = 2; };

// Geometry and per-strip-block companion lists of one launch.
struct Geom {
    int strips;        // strips across the grid
    int nitems;        // strip blocks
    const int* items;  // strip block t: strip items[4t], rows items[4t + 1] .. items[4t + 2] - 1,
                       // items[4t + 3] = 1 for a plain interior block (the fast path)
    const int* gstart; // nodes with a bounce-back link of item t: glist[gstart[t] .. gstart[t + 1]), or nullptr
    const int* glist;  // (j * nx + i)
    const int* dstart; // Dirichlet nodes of item t: dlist[dstart[t] .. dstart[t + 1]), or nullptr (not fused)
    const DirNode* dlist;
    const double* D64;
    DirValues bv;
};

template <typename T>
struct Pair {  // a lane's node pair of one row, as loaded
    using V2 = typename Vec2<T>::type;
    V2 e, u, v, d;
    uint32_t types;  // bits 0-15: type bytes of the two columns; bits 16-17 / 18-19: mirror flags
};

template <typename T>
struct SrcP {  // source quantities of the pair (x: column 0, y: column 1)
    using V2 = typename Vec2<T>::type;
    V2 eta, D, o1, o2, o3, o4, o5, o6, o7, o8, ownh, hFx, hFy;
};

// FP32 coefficients as lane pairs (FP64 does not use them)
template <typename T>
__device__ __forceinline__ Coef2 pairs_of(const Coef<T>& c)
{
    if constexpr (std::is_same<T, float>::value) return coef2_of(c);
    else return Coef2{};
}

template <typename T, int FM>
__device__ __forceinline__ void derive_pair(const Coef<T>& c, const Coef2& c2, const Pair<T>& p, SrcP<T>& s)
{
    const Raw<T> r0{p.e.x, p.u.x, p.v.x, p.d.x, (uint8_t)((p.types >> 16) & 3)};
    const Raw<T> r1{p.e.y, p.u.y, p.v.y, p.d.y, (uint8_t)((p.types >> 18) & 3)};
#ifndef MACLAB_MARCH_SCALAR_DERIVE
    if constexpr (std::is_same<T, float>::value) {
#else
    if constexpr (false) {
#endif
        Src2 q;
        derive2<FM>(c2, r0, r1, q);
        s.eta = q.eta; s.D = q.D; s.o1 = q.o1; s.o2 = q.o2; s.o3 = q.o3; s.o4 = q.o4; s.o5 = q.o5;
        s.o6 = q.o6; s.o7 = q.o7; s.o8 = q.o8; s.ownh = q.ownh; s.hFx = q.hFx; s.hFy = q.hFy;
    } else {
        Src<T> a, b;
        derive<T, FM>(c, r0, a);
        derive<T, FM>(c, r1, b);
        using V2 = typename Vec2<T>::type;
        s.eta = V2{a.eta, b.eta}; s.D = V2{a.D, b.D};
        s.o1 = V2{a.o1, b.o1}; s.o2 = V2{a.o2, b.o2}; s.o3 = V2{a.o3, b.o3}; s.o4 = V2{a.o4, b.o4};
        s.o5 = V2{a.o5, b.o5}; s.o6 = V2{a.o6, b.o6}; s.o7 = V2{a.o7, b.o7}; s.o8 = V2{a.o8, b.o8};
        s.ownh = V2{a.ownh, b.ownh}; s.hFx = V2{a.hFx, b.hFx}; s.hFy = V2{a.hFy, b.hFy};
    }
}

// Column sources of a lane, fixed for the whole strip: the two columns
// resolved through the W / E edge kinds (-1 behind a bounce-back edge) with
// their mirror flags; vec when they are the in-grid pair x, x + 1.
struct LaneCols2 {
    int c0, c1;
    uint32_t flips;  // x-mirror flag of column 0 at bit 16, column 1 at bit 18
    bool vec;
};

template <typename T>
__device__ __forceinline__ LaneCols2 lane_cols(const Fields<T>& f, int x)
{
    LaneCols2 lc;
    uint8_t f0 = 0, f1 = 0;
    lc.c0 = resolve_index(x, f.nx, f.edge[0], f.edge[1], 1, f0);
    lc.c1 = resolve_index(x + 1, f.nx, f.edge[0], f.edge[1], 1, f1);
    lc.flips = ((uint32_t)f0 << 16) | ((uint32_t)f1 << 18);
    lc.vec = x >= 0 && x + 2 <= f.nx;
    return lc;
}

// Shared memory of one warp.  Raw rows are lane-private (each lane reads
// back only what its own copies wrote, so cp.async.wait_group orders them);
// derived rows are shared by the warp (__syncwarp orders them).  Derived
// values are split by column parity: even columns X0 + 2j at [0][1 + j],
// odd columns X0 + 2j + 1 at [1][1 + j], so that a warp reading one column
// per lane touches consecutive words (no bank conflicts), and the reads of
// lanes 0 and 31 one column outside the strip stay inside the arrays.
constexpr int RAW_SLOTS = AHEAD + 1;  // 3: the same period as the derived rows
template <typename T>
struct WarpSmem {
    using V2 = typename Vec2<T>::type;
    V2 raw[RAW_SLOTS][4][32];        // eta, u, v, D of each lane's pair
    uint32_t rtype[RAW_SLOTS][32][2];  // the aligned 4-byte type words holding the pair's bytes
    T o[3][4][2][34];           // o1, o2, o4, o5 by column parity
    V2 o3[3][32];               // o3 of each lane's pair
    V2 ed[3][2][34];            // (eta, D) by column parity
};
template <typename T>
__host__ __device__ constexpr size_t smem_bytes() { return WARPS * sizeof(WarpSmem<T>); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int BYTES>
__device__ __forceinline__ void cp_async_z(uint32_t dst, const void* src, bool valid)
{
    // src-size 0 zero-fills the destination (a source behind a wall)
    if (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0));
    else if (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 8 : 0));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0));
}

// Issue the copies of the lane's pair of row y into raw slot `slot` (one
// commit group).  EDGE = false: a plain interior strip block (it reads
// inside the grid with 32-bit offsets, and the nodes it writes are fluid or
// Dirichlet nodes without a bounce-back link, so no node type is needed).
// EDGE = true: any strip block; a row outside the grid is resolved
// through the S / N edge kinds (the same for the whole warp), the lane's
// columns through its fixed sources; sources behind a wall read zero.
template <typename T, bool EDGE, typename SM = WarpSmem<T>>
__device__ __forceinline__ void fetch_row(const Fields<T>& f, int y, int x, const LaneCols2& lc, SM& sm, int slot,
                                          int lane)
{
    const T* fld[4] = {f.eta, f.u, f.v, f.D};
    const uint32_t dst = smem_addr(&sm.raw[slot][0][lane]);
    constexpr uint32_t FS = 32 * sizeof(typename Vec2<T>::type);  // bytes between fields of a slot
    int rr = y;
    if (EDGE && (y < 0 || y >= f.ny)) {
        uint8_t fy = 0;
        rr = resolve_index(y, f.ny, f.edge[2], f.edge[3], 2, fy);
    }
    if (!EDGE || (rr >= 0 && lc.vec)) {
        const size_t off = EDGE ? (size_t)rr * f.pitch + x : (size_t)(unsigned)(y * f.pitch + x);
#pragma unroll
        for (int q = 0; q < 4; ++q) cp_async_z<2 * sizeof(T)>(dst + q * FS, fld[q] + off, true);
        // the type bytes of x, x + 1 lie in the aligned word at off & ~3
        // (plain interior blocks do not need them)
        if constexpr (EDGE) cp_async_z<4>(smem_addr(&sm.rtype[slot][lane][0]), f.type + (off & ~(size_t)3), true);
    } else {
        const bool ok0 = rr >= 0 && lc.c0 >= 0, ok1 = rr >= 0 && lc.c1 >= 0;
        const size_t row = rr >= 0 ? (size_t)rr * f.pitch : 0;
        const size_t i0 = ok0 ? row + lc.c0 : 0, i1 = ok1 ? row + lc.c1 : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cp_async_z<sizeof(T)>(dst + q * FS, fld[q] + i0, ok0);
            cp_async_z<sizeof(T)>(dst + q * FS + sizeof(T), fld[q] + i1, ok1);
        }
        if constexpr (EDGE) {
            const uint32_t tdst = smem_addr(&sm.rtype[slot][lane][0]);
            cp_async_z<4>(tdst, f.type + (i0 & ~(size_t)3), ok0);
            cp_async_z<4>(tdst + 4, f.type + (i1 & ~(size_t)3), ok1);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
}

// Read back the lane's staged pair of row y (its copies complete).
template <typename T, bool EDGE, typename SM = WarpSmem<T>>
__device__ __forceinline__ void read_row(const Fields<T>& f, int y, int x, const LaneCols2& lc, const SM& sm, int slot,
                                         int lane, Pair<T>& p)
{
    p.e = sm.raw[slot][0][lane];
    p.u = sm.raw[slot][1][lane];
    p.v = sm.raw[slot][2][lane];
    p.d = sm.raw[slot][3][lane];
    if constexpr (!EDGE) {
        p.types = 0;  // plain interior block: fluid or Dirichlet nodes only, no mirrors
        return;
    } else {
    uint8_t fy = 0;
    int rr = y;
    if (y < 0 || y >= f.ny) rr = resolve_index(y, f.ny, f.edge[2], f.edge[3], 2, fy);
    if (rr >= 0 && lc.vec) {
        p.types = ((sm.rtype[slot][lane][0] >> (8 * (x & 3))) & 0xffffu) | ((uint32_t)fy << 16) |
                  ((uint32_t)fy << 18);
        return;
    }
    uint32_t t = 0;
    if (rr >= 0 && lc.c0 >= 0)
        t |= ((sm.rtype[slot][lane][0] >> (8 * (lc.c0 & 3))) & 0xffu) | (lc.flips & (3u << 16)) | ((uint32_t)fy << 16);
    if (rr >= 0 && lc.c1 >= 0)
        t |= (((sm.rtype[slot][lane][1] >> (8 * (lc.c1 & 3))) & 0xffu) << 8) | (lc.flips & (3u << 18)) |
             ((uint32_t)fy << 18);
    p.types = t;
    }
}

template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_dn1(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// The node's own quantities of an output row, carried from its derivation
// to its update one row later.
template <typename T>
struct Own {
    typename Vec2<T>::type ownh, hFx, hFy;
    uint32_t types;
};

// The update of the lane's two receivers (x, x + 1) of an output row, FP32:
// the (eta, D) stencils of each receiver as in update_tail, then the
// streamed sums and the update with one receiver per lane of the paired
// instructions.  Each lane takes the operations of streamed_sums and
// update_tail in their order, so the results are bitwise those of the
// scalar form.  Operands are receiver pairs (.x for x, .y for x + 1):
// A1 = cL_o1, M2 = mL_o2, C5 = cR_o5, M4 = mR_o4, M3 = mC_o3, P8 = pL_o8,
// P6 = pR_o6, P7 = pC_o7; m, c, p hold (eta, D) at columns x - 1 .. x + 2
// of the rows above, own and below.
__device__ __forceinline__ void gather_pair(const Coef2& K, float2 A1, float2 M2, float2 C5, float2 M4,
                                            float2 M3, float2 P8, float2 P6, float2 P7, const float2 (&m)[4],
                                            const float2 (&c)[4], const float2 (&p)[4], float2 ownh, float2 hFx,
                                            float2 hFy, bool ns0, bool ns1, float2& oe, float2& ou, float2& ov)
{
    using P = Op2;
    const float2 z = K.nz, q2 = splat(0.25f);
    float2 S[2], X[2], Y[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float2 mL = m[k], mC = m[k + 1], mR = m[k + 2], cL = c[k], cR = c[k + 2];
        const float2 pL = p[k], pC = p[k + 1], pR = p[k + 2];
        const float2 ML = P::fma(q2, P::add(mL, pL), cL), MR = P::fma(q2, P::add(mR, pR), cR);
        S[k] = P::add(P::add(ML, MR), P::add(mC, pC));
        X[k] = P::sub(ML, MR);
        Y[k] = P::fma(q2, P::sub(P::add(mL, mR), P::add(pL, pR)), P::sub(mC, pC));
    }
    // regroup by receiver: eta stencils (.x of each) and D stencils (.y)
    const float2 SE = make_float2(S[0].x, S[1].x), SD = make_float2(S[0].y, S[1].y);
    const float2 XE = make_float2(X[0].x, X[1].x), XD = make_float2(X[0].y, X[1].y);
    const float2 YE = make_float2(Y[0].x, Y[1].x), YD = make_float2(Y[0].y, Y[1].y);
    const float2 E = make_float2(c[1].x, c[2].x), D = make_float2(c[1].y, c[2].y);
    // streamed sums
    const float2 a1 = P::add(A1, M2), a2 = P::add(C5, M4), sym = P::add(P::add(M2, M4), M3);
    const float2 OL = P::add(a1, P8), OR = P::add(a2, P6);
    const float2 Sh = P::add(P::add(OL, OR), P::add(M3, P7));
    const float2 Sx = P::sub(OL, OR);
    const float2 Sy = P::sub(sym, P::add(P::add(P8, P6), P7));
    // update: -B = round(-G6 eta), the negated rounded product
    const float2 A = P::mul(K.G6, D, z), nB = P::mul(K.nG6, E, z);
    oe = P::add(P::add(ownh, Sh), P::fma(A, SE, P::mul(nB, SD, z)));
    const float2 e2 = K.e;
    const float2 hu = P::fma(e2, P::add(Sx, P::fma(A, XE, P::mul(nB, XD, z))), hFx);
    const float2 hv = P::fma(e2, P::add(Sy, P::fma(A, YE, P::mul(nB, YD, z))), hFy);
    const float2 h = P::add(D, oe);
    const float2 inv = make_float2(Op<float>::rcp(h.x), Op<float>::rcp(h.y));
    ou = P::mul(hu, inv, z);
    ov = P::mul(hv, inv, z);
    if (ns0) ou.x = 0.f, ov.x = 0.f;
    if (ns1) ou.y = 0.f, ov.y = 0.f;
}

// Row r: issue the copies of row r + 2, derive row r into derived slot sp
// (after every lane has finished reading that slot), then (when DONE)
// update output row r - 1 from the derived slots sm_ (row r - 2), sc (row
// r - 1) and sp (row r, partly still in registers).  Raw and derived rows
// share the period 3: row r's raw slot is sp, and row r + 2 is copied into
// raw slot sc (freed by row r - 1).
// FR (a fringe pass, EDGE only): output rows fr0 and fr1 and the lane's
// columns in fcol are a one-node fringe around the strip block; a fringe
// node is written only if it is a fluid or no-slip node (its own strip
// block writes a Dirichlet node).
template <typename T, int FM, bool EDGE, bool FR = false>
__device__ __forceinline__ void march_row(const Fields<T>& f, int r, int x, const LaneCols2& lc, int last,
                                          unsigned colmask, int lane, WarpSmem<T>& sm, const Coef2& c2, int sp,
                                          int sc, int sm_,
                                          Own<T>& own, bool done, typename Vec2<T>::type (&o3r)[3],
                                          typename Vec2<T>::type (&edr)[3][2], int fr0 = 0, int fr1 = 0,
                                          unsigned fcol = 0)
{
    using V2 = typename Vec2<T>::type;
    Pair<T> p;
    if (r + AHEAD <= last) fetch_row<T, EDGE>(f, r + AHEAD, x, lc, sm, sc, lane);
    else asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(AHEAD));
    read_row<T, EDGE>(f, r, x, lc, sm, sp, lane, p);
    SrcP<T> d;
    derive_pair<T, FM>(f.c, c2, p, d);
    __syncwarp();  // every lane has read derived slot sp (row r - 3) for the last time
    {
        const V2 ov4[4] = {d.o1, d.o2, d.o4, d.o5};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sm.o[sp][q][0][1 + lane] = ov4[q].x;
            sm.o[sp][q][1][1 + lane] = ov4[q].y;
        }
        if (CARRY == 0) sm.o3[sp][lane] = d.o3;
        sm.ed[sp][0][1 + lane] = V2{d.eta.x, d.D.x};
        sm.ed[sp][1][1 + lane] = V2{d.eta.y, d.D.y};
    }
    const T Lo8 = shfl_up1(d.o8.y), Ro6 = shfl_dn1(d.o6.x);
    __syncwarp();  // derived slot sp is visible to the warp
    if (done) {
        // output row r - 1: its own row in slot sc, the row above in sm_, the row below r
        const V2 m[4] = {sm.ed[sm_][1][lane], CARRY >= 2 ? edr[sm_][0] : sm.ed[sm_][0][1 + lane],
                         CARRY >= 2 ? edr[sm_][1] : sm.ed[sm_][1][1 + lane], sm.ed[sm_][0][2 + lane]};
        const V2 c[4] = {sm.ed[sc][1][lane], CARRY >= 2 ? edr[sc][0] : sm.ed[sc][0][1 + lane],
                         CARRY >= 2 ? edr[sc][1] : sm.ed[sc][1][1 + lane], sm.ed[sc][0][2 + lane]};
        const V2 pe[4] = {sm.ed[sp][1][lane], V2{d.eta.x, d.D.x}, V2{d.eta.y, d.D.y}, sm.ed[sp][0][2 + lane]};
        // o2 at x - 1, x; o4 at x + 1, x + 2; o3 at x, x + 1 (row above); o1 at x - 1, x; o5 at x + 1, x + 2
        // (column x - 1 is odd column j = lane - 1, x + 2 even column j = lane + 1)
        const V2 M2 = V2{sm.o[sm_][1][1][lane], sm.o[sm_][1][0][1 + lane]};
        const V2 M4 = V2{sm.o[sm_][2][1][1 + lane], sm.o[sm_][2][0][2 + lane]};
        const V2 M3 = CARRY >= 1 ? o3r[sm_] : sm.o3[sm_][lane];
        const V2 A1 = V2{sm.o[sc][0][1][lane], sm.o[sc][0][0][1 + lane]};
        const V2 C5 = V2{sm.o[sc][3][1][1 + lane], sm.o[sc][3][0][2 + lane]};
        // written: node kinds 1 .. 7 without the bounce-back bit (type byte in
        // 1 .. 7); a plain interior block has only such nodes and no no-slip ones
        const uint32_t k0 = own.types & 0xffu, k1 = (own.types >> 8) & 0xffu;
        unsigned ok = EDGE ? colmask & ((k0 - 1u < 7u ? 1u : 0u) | (k1 - 1u < 7u ? 2u : 0u)) : colmask;
        if (FR) {
            const unsigned fr = (r - 1 == fr0 || r - 1 == fr1) ? 3u : fcol;
            const unsigned dir = (k0 - (unsigned)K_DIR_H < 3u ? 1u : 0u) | (k1 - (unsigned)K_DIR_H < 3u ? 2u : 0u);
            ok &= ~(fr & dir);
            if (r - 1 < 0 || r - 1 >= f.ny) ok = 0;  // a fringe row beyond the grid edge
        }
        const bool ns0 = EDGE && (k0 & KIND_MASK) == K_NOSLIP, ns1 = EDGE && (k1 & KIND_MASK) == K_NOSLIP;
        V2 oe, ou, ov;
        if constexpr (std::is_same<T, float>::value) {
            gather_pair(c2, A1, M2, C5, M4, M3, V2{Lo8, d.o8.x}, V2{d.o6.y, Ro6}, d.o7, m, c, pe, own.ownh,
                        own.hFx, own.hFy, ns0, ns1, oe, ou, ov);
        } else {
            using O = Op<T>;
            T Sh, Sx, Sy;
            streamed_sums<T>(O::add(A1.x, M2.x), O::add(C5.x, M4.x), O::add(O::add(M2.x, M4.x), M3.x), M3.x, Lo8,
                             d.o6.y, d.o7.x, Sh, Sx, Sy);
            update_tail<T>(f.c, Sh, Sx, Sy, m[0], m[1], m[2], c[0], c[2], pe[0], pe[1], pe[2], c[1].x, c[1].y,
                           own.ownh.x, own.hFx.x, own.hFy.x, ns0, oe.x, ou.x, ov.x);
            streamed_sums<T>(O::add(A1.y, M2.y), O::add(C5.y, M4.y), O::add(O::add(M2.y, M4.y), M3.y), M3.y,
                             d.o8.x, Ro6, d.o7.y, Sh, Sx, Sy);
            update_tail<T>(f.c, Sh, Sx, Sy, m[1], m[2], m[3], c[1], c[3], pe[1], pe[2], pe[3], c[2].x, c[2].y,
                           own.ownh.y, own.hFx.y, own.hFy.y, ns1, oe.y, ou.y, ov.y);
        }
        const size_t idx = EDGE ? (size_t)(r - 1) * f.pitch + x : (size_t)(unsigned)((r - 1) * f.pitch + x);
        if (!EDGE && OUT == 60) {
            // plain interior block, lanes 0 and 31 pure halo: both columns or none
            if (ok) {
                *reinterpret_cast<V2*>(f.eta1 + idx) = oe;
                *reinterpret_cast<V2*>(f.u1 + idx) = ou;
                *reinterpret_cast<V2*>(f.v1 + idx) = ov;
            }
        } else if (ok == 3u) {
            *reinterpret_cast<V2*>(f.eta1 + idx) = oe;
            *reinterpret_cast<V2*>(f.u1 + idx) = ou;
            *reinterpret_cast<V2*>(f.v1 + idx) = ov;
        } else if (ok) {
            // one column: selects, not a runtime array index (which would
            // put the values in local memory)
            const bool hi = ok == 2u;
            const size_t i = idx + (hi ? 1 : 0);
            f.eta1[i] = hi ? oe.y : oe.x;
            f.u1[i] = hi ? ou.y : ou.x;
            f.v1[i] = hi ? ov.y : ov.x;
        }
    }
    own.ownh = d.ownh;
    own.hFx = d.hFx;
    own.hFy = d.hFy;
    own.types = p.types;
    if (CARRY >= 1) o3r[sp] = d.o3;
    if (CARRY >= 2) {
        edr[sp][0] = V2{d.eta.x, d.D.x};
        edr[sp][1] = V2{d.eta.y, d.D.y};
    }
}

// Rows j0 .. j1 - 1 of strip s (derived rows j0 - 1 .. j1).  FR: a
// fringe pass, which also writes local columns 1 and 62 and whose rows
// j0 and j1 - 1 are the fringe (see march_row).
template <typename T, int FM, bool EDGE, bool FR = false>
__device__ __forceinline__ void march_strip(const Fields<T>& f, const Coef2& c2, int s, int j0, int j1, int lane,
                                            WarpSmem<T>& sm)
{
    const int x = first_col(s) + 2 * lane;
    // the lane's columns that the strip writes and that lie in the grid
    constexpr int LO = FR ? 1 : 1 + HALF, HI = FR ? 62 : 62 - HALF;
    unsigned colmask = (2 * lane >= LO && 2 * lane <= HI ? 1u : 0u) | (2 * lane + 1 >= LO && 2 * lane + 1 <= HI ? 2u : 0u);
    // fringe columns: local 1 (lane 0, second column) and 62 (lane 31,
    // first column), derived but not written by a 60-column strip
    static_assert(!FR || HALF == 1, "a fringe pass needs 60-column strips");
    const unsigned fcol = FR ? ((lane == 0 ? 2u : 0u) | (lane == 31 ? 1u : 0u)) : 0u;
    LaneCols2 lc{x, x + 1, 0u, true};
    if (EDGE) {
        lc = lane_cols(f, x);
        if (x < 0 || x >= f.nx) colmask &= ~1u;
        if (x + 1 < 0 || x + 1 >= f.nx) colmask &= ~2u;
    }
    const int last = j1;
    // rows j0 - 1 and j0 in flight in raw slots 0 and 1
#pragma unroll
    for (int q = 0; q < AHEAD; ++q) {
        if (j0 - 1 + q <= last) fetch_row<T, EDGE>(f, j0 - 1 + q, x, lc, sm, q, lane);
        else asm volatile("cp.async.commit_group;\n" ::);
    }
    Own<T> own;
    typename Vec2<T>::type o3r[3], edr[3][2];  // carried in registers (CARRY)
    // rows rotate through slots: row r in raw and derived slot (r - j0 + 1) % 3
    march_row<T, FM, EDGE, FR>(f, j0 - 1, x, lc, last, colmask, lane, sm, c2, 0, 2, 1, own, false, o3r, edr, j0, j1 - 1, fcol);
    march_row<T, FM, EDGE, FR>(f, j0, x, lc, last, colmask, lane, sm, c2, 1, 0, 2, own, false, o3r, edr, j0, j1 - 1, fcol);
    for (int r = j0 + 1;; r += 3) {
        march_row<T, FM, EDGE, FR>(f, r, x, lc, last, colmask, lane, sm, c2, 2, 1, 0, own, true, o3r, edr, j0, j1 - 1, fcol);
        if (r >= last) break;
        march_row<T, FM, EDGE, FR>(f, r + 1, x, lc, last, colmask, lane, sm, c2, 0, 2, 1, own, true, o3r, edr, j0, j1 - 1, fcol);
        if (r + 1 >= last) break;
        march_row<T, FM, EDGE, FR>(f, r + 2, x, lc, last, colmask, lane, sm, c2, 1, 0, 2, own, true, o3r, edr, j0, j1 - 1, fcol);
        if (r + 2 >= last) break;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}


// ---------------------------------------------------------------------------
// Two steps per pass (temporal blocking, FP32, plain strip blocks whose
// rows j0 - 2 .. j1 + 1 and 64 columns lie inside the grid and hold only
// fluid nodes).  Level 1 is the row march above: derive row r (state n),
// update row r - 1 to state n + 1, but in registers only.  Level 2 derives
// that row again from those registers into a second ring and, one row
// behind, updates row r - 2 to state n + 2 and stores it.  Level 1 is valid
// on local columns 1 .. 62 (it needs a derived column either side), level 2
// on 2 .. 61, the 60 columns a strip writes.  Every node takes the
// operations of two single steps in their order, so the result is bitwise
// that of two single steps.
struct Ring {
    float o[3][4][2][34];  // o1, o2, o4, o5 by column parity
    float2 ed[3][2][34];   // (eta, D) by column parity
};
struct WarpSmem2 {
    float2 raw[RAW_SLOTS][4][32];  // raw staging (plain blocks: no type words)
    Ring a;                        // level 1 (o3 and the lane's own (eta, D) in registers)
    Ring b;                        // level 2
};
__host__ __device__ constexpr size_t smem2_bytes() { return WARPS * sizeof(WarpSmem2); }

template <int FM>
__device__ __forceinline__ void march2_row(const Fields<float>& f, int r, int x, int last, int lane, WarpSmem2& sm,
                                           const Coef2& c2, int sp, int sc, int sm_, Own<float>& own1,
                                           Own<float>& own2, bool lv1, bool lv2, float2 (&o3a)[3], float2 (&eda)[3][2],
                                           float2 (&o3b)[3], float2 (&edb)[3][2])
{
    Ring& A = sm.a;
    Ring& B = sm.b;
    const LaneCols2 lc{x, x + 1, 0u, true};
    Pair<float> p;
    if (r + AHEAD <= last) fetch_row<float, false, WarpSmem2>(f, r + AHEAD, x, lc, sm, sc, lane);
    else asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group %0;\n" ::"n"(AHEAD));
    read_row<float, false, WarpSmem2>(f, r, x, lc, sm, sp, lane, p);
    SrcP<float> d;
    derive_pair<float, FM>(f.c, c2, p, d);
    __syncwarp();  // every lane is done with level-1 slot sp (row r - 3) and level-2 slot sc (row r - 4)
    {
        const float2 ov4[4] = {d.o1, d.o2, d.o4, d.o5};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            A.o[sp][q][0][1 + lane] = ov4[q].x;
            A.o[sp][q][1][1 + lane] = ov4[q].y;
        }
        A.ed[sp][0][1 + lane] = float2{d.eta.x, d.D.x};
        A.ed[sp][1][1 + lane] = float2{d.eta.y, d.D.y};
    }
    const float Lo8 = shfl_up1(d.o8.y), Ro6 = shfl_dn1(d.o6.x);
    __syncwarp();
    if (lv1) {
        // level 1: row r - 1 to state n + 1 (own row in slot sc, above sm_, below r)
        const float2 m[4] = {A.ed[sm_][1][lane], eda[sm_][0], eda[sm_][1], A.ed[sm_][0][2 + lane]};
        const float2 c[4] = {A.ed[sc][1][lane], eda[sc][0], eda[sc][1], A.ed[sc][0][2 + lane]};
        const float2 pe[4] = {A.ed[sp][1][lane], float2{d.eta.x, d.D.x}, float2{d.eta.y, d.D.y}, A.ed[sp][0][2 + lane]};
        const float2 M2 = float2{A.o[sm_][1][1][lane], A.o[sm_][1][0][1 + lane]};
        const float2 M4 = float2{A.o[sm_][2][1][1 + lane], A.o[sm_][2][0][2 + lane]};
        const float2 A1 = float2{A.o[sc][0][1][lane], A.o[sc][0][0][1 + lane]};
        const float2 C5 = float2{A.o[sc][3][1][1 + lane], A.o[sc][3][0][2 + lane]};
        float2 oe, ou, ov;
        gather_pair(c2, A1, M2, C5, M4, o3a[sm_], float2{Lo8, d.o8.x}, float2{d.o6.y, Ro6}, d.o7, m, c, pe, own1.ownh,
                    own1.hFx, own1.hFy, false, false, oe, ou, ov);
        // level 2: derive row r - 1 of state n + 1 into slot sc
        Pair<float> q;
        q.e = oe;
        q.u = ou;
        q.v = ov;
        q.d = float2{c[1].y, c[2].y};
        q.types = 0;
        SrcP<float> d2;
        derive_pair<float, FM>(f.c, c2, q, d2);
        {
            const float2 ov4[4] = {d2.o1, d2.o2, d2.o4, d2.o5};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                B.o[sc][k][0][1 + lane] = ov4[k].x;
                B.o[sc][k][1][1 + lane] = ov4[k].y;
            }
            B.ed[sc][0][1 + lane] = float2{d2.eta.x, d2.D.x};
            B.ed[sc][1][1 + lane] = float2{d2.eta.y, d2.D.y};
        }
        const float Lo8b = shfl_up1(d2.o8.y), Ro6b = shfl_dn1(d2.o6.x);
        __syncwarp();  // level-2 slot sc is visible to the warp
        if (lv2) {
            // level 2: row r - 2 to state n + 2 (own row in slot sm_, above sp, below r - 1)
            const float2 mb[4] = {B.ed[sp][1][lane], edb[sp][0], edb[sp][1], B.ed[sp][0][2 + lane]};
            const float2 cb[4] = {B.ed[sm_][1][lane], edb[sm_][0], edb[sm_][1], B.ed[sm_][0][2 + lane]};
            const float2 pb[4] = {B.ed[sc][1][lane], float2{d2.eta.x, d2.D.x}, float2{d2.eta.y, d2.D.y},
                                  B.ed[sc][0][2 + lane]};
            const float2 M2b = float2{B.o[sp][1][1][lane], B.o[sp][1][0][1 + lane]};
            const float2 M4b = float2{B.o[sp][2][1][1 + lane], B.o[sp][2][0][2 + lane]};
            const float2 A1b = float2{B.o[sm_][0][1][lane], B.o[sm_][0][0][1 + lane]};
            const float2 C5b = float2{B.o[sm_][3][1][1 + lane], B.o[sm_][3][0][2 + lane]};
            float2 oe2, ou2, ov2;
            gather_pair(c2, A1b, M2b, C5b, M4b, o3b[sp], float2{Lo8b, d2.o8.x}, float2{d2.o6.y, Ro6b}, d2.o7, mb, cb,
                        pb, own2.ownh, own2.hFx, own2.hFy, false, false, oe2, ou2, ov2);
            // lanes 0 and 31 only supply neighbours (60 written columns)
            if (lane >= 1 && lane <= 30) {
                const size_t idx = (size_t)(unsigned)((r - 2) * f.pitch + x);
                *reinterpret_cast<float2*>(f.eta1 + idx) = oe2;
                *reinterpret_cast<float2*>(f.u1 + idx) = ou2;
                *reinterpret_cast<float2*>(f.v1 + idx) = ov2;
            }
        }
        own2.ownh = d2.ownh;
        own2.hFx = d2.hFx;
        own2.hFy = d2.hFy;
        o3b[sc] = d2.o3;
        edb[sc][0] = float2{d2.eta.x, d2.D.x};
        edb[sc][1] = float2{d2.eta.y, d2.D.y};
    }
    own1.ownh = d.ownh;
    own1.hFx = d.hFx;
    own1.hFy = d.hFy;
    o3a[sp] = d.o3;
    eda[sp][0] = float2{d.eta.x, d.D.x};
    eda[sp][1] = float2{d.eta.y, d.D.y};
}

// Rows j0 .. j1 - 1 of strip s at state n + 2 (derived rows j0 - 2 .. j1 + 1
// of state n, level-1 rows j0 - 1 .. j1).
template <int FM>
__device__ __forceinline__ void march_strip2(const Fields<float>& f, const Coef2& c2, int s, int j0, int j1, int lane,
                                             WarpSmem2& sm)
{
    static_assert(HALF == 1, "two levels need 60-column strips");
    const int x = first_col(s) + 2 * lane;
    const LaneCols2 lc{x, x + 1, 0u, true};
    const int last = j1 + 1;
#pragma unroll
    for (int q = 0; q < AHEAD; ++q) fetch_row<float, false, WarpSmem2>(f, j0 - 2 + q, x, lc, sm, q, lane);
    Own<float> own1, own2;
    float2 o3a[3], eda[3][2], o3b[3], edb[3][2];
    // row r in slot (r - j0 + 2) % 3
    march2_row<FM>(f, j0 - 2, x, last, lane, sm, c2, 0, 2, 1, own1, own2, false, false, o3a, eda, o3b, edb);
    march2_row<FM>(f, j0 - 1, x, last, lane, sm, c2, 1, 0, 2, own1, own2, false, false, o3a, eda, o3b, edb);
    march2_row<FM>(f, j0, x, last, lane, sm, c2, 2, 1, 0, own1, own2, true, false, o3a, eda, o3b, edb);
    march2_row<FM>(f, j0 + 1, x, last, lane, sm, c2, 0, 2, 1, own1, own2, true, false, o3a, eda, o3b, edb);
    for (int r = j0 + 2;; r += 3) {
        march2_row<FM>(f, r, x, last, lane, sm, c2, 1, 0, 2, own1, own2, true, true, o3a, eda, o3b, edb);
        if (r >= last) break;
        march2_row<FM>(f, r + 1, x, last, lane, sm, c2, 2, 1, 0, own1, own2, true, true, o3a, eda, o3b, edb);
        if (r + 1 >= last) break;
        march2_row<FM>(f, r + 2, x, last, lane, sm, c2, 0, 2, 1, own1, own2, true, true, o3a, eda, o3b, edb);
        if (r + 2 >= last) break;
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

}  // namespace march

// Strip block t = (strip t % strips, row block t / strips) per warp.
template <typename T, int FM>
__global__ void __launch_bounds__(march::THREADS, march::MinBlocks<T>::value)
step_march_kernel(const __grid_constant__ Fields<T> f, const __grid_constant__ march::Geom g)
{
    extern __shared__ __align__(16) unsigned char march_smem[];
    const int lane = threadIdx.x & 31, wib = (int)(threadIdx.x >> 5);
    march::WarpSmem<T>& sm = reinterpret_cast<march::WarpSmem<T>*>(march_smem)[wib];
    const int item = (int)blockIdx.x * march::WARPS + wib;
    if (item >= g.nitems) return;  // whole warp
    const int4 t = reinterpret_cast<const int4*>(g.items)[item];
    const int s = t.x, j0 = t.y, j1 = t.z;
    if (t.w) march::march_strip<T, FM, false>(f, march::pairs_of(f.c), s, j0, j1, lane, sm);
    else march::march_strip<T, FM, true>(f, march::pairs_of(f.c), s, j0, j1, lane, sm);
    if (g.gstart) {
        const int e = g.gstart[item + 1];
        for (int k = g.gstart[item] + lane; k < e; k += 32) {
            const int node = g.glist[k];
            general_node<T>(f, node % f.nx, node / f.nx);
        }
    }
    if (g.dstart) {
        const int b = g.dstart[item], e = g.dstart[item + 1];
        if (b < e) {
            __syncwarp();  // the strip block's new values are visible to the warp
            for (int k = b + lane; k < e; k += 32)
                dirichlet_node(f.eta1, f.u1, f.v1, f.D, g.D64, g.dlist[k], g.bv);
        }
    }
}

}  // namespace maclab

namespace maclab {

// Two steps of the strip blocks sel[0 .. n) (plain, see march_strip2) from
// (eta, u, v) to (eta1, u1, v1).
template <int FM>
__global__ void __launch_bounds__(march::THREADS, 4)
step_march2_kernel(const __grid_constant__ Fields<float> f, const int* __restrict__ items, const int* __restrict__ sel,
                   int n)
{
    extern __shared__ __align__(16) unsigned char march_smem[];
    const int lane = threadIdx.x & 31, wib = (int)(threadIdx.x >> 5);
    march::WarpSmem2& sm = reinterpret_cast<march::WarpSmem2*>(march_smem)[wib];
    const int k = (int)blockIdx.x * march::WARPS + wib;
    if (k >= n) return;  // whole warp
    const int4 t = reinterpret_cast<const int4*>(items)[sel[k]];
    march::march_strip2<FM>(f, march::pairs_of(f.c), t.x, t.y, t.z, lane, sm);
}

// One step of the strip blocks sel[0 .. n), with their nodes with a
// bounce-back link and (fused) Dirichlet nodes.  FR: the strip blocks also
// write a one-node fringe (rows j0 - 1 and j1, local columns 1 and 62; its
// Dirichlet nodes excepted), so that a second step of the same strip blocks
// finds every neighbour it reads at the middle state.
template <int FM, bool FR>
__global__ void __launch_bounds__(march::THREADS, march::MinBlocks<float>::value)
step_march_list_kernel(const __grid_constant__ Fields<float> f, const __grid_constant__ march::Geom g,
                       const int* __restrict__ sel, int n)
{
    extern __shared__ __align__(16) unsigned char march_smem[];
    const int lane = threadIdx.x & 31, wib = (int)(threadIdx.x >> 5);
    march::WarpSmem<float>& sm = reinterpret_cast<march::WarpSmem<float>*>(march_smem)[wib];
    const int k = (int)blockIdx.x * march::WARPS + wib;
    if (k >= n) return;  // whole warp
    const int item = sel[k];
    const int4 t = reinterpret_cast<const int4*>(g.items)[item];
    const int s = t.x, j0 = t.y, j1 = t.z;
    if (FR) march::march_strip<float, FM, true, true>(f, march::pairs_of(f.c), s, j0 - 1, j1 + 1, lane, sm);
    else if (t.w) march::march_strip<float, FM, false>(f, march::pairs_of(f.c), s, j0, j1, lane, sm);
    else march::march_strip<float, FM, true>(f, march::pairs_of(f.c), s, j0, j1, lane, sm);
    if (g.gstart) {
        const int e = g.gstart[item + 1];
        for (int q = g.gstart[item] + lane; q < e; q += 32) {
            const int node = g.glist[q];
            general_node<float>(f, node % f.nx, node / f.nx);
        }
    }
    if (g.dstart) {
        const int b = g.dstart[item], e = g.dstart[item + 1];
        if (b < e) {
            __syncwarp();  // the strip block's new values are visible to the warp
            for (int q = b + lane; q < e; q += 32)
                dirichlet_node(f.eta1, f.u1, f.v1, f.D, g.D64, g.dlist[q], g.bv);
        }
    }
}

}  // namespace maclab
