// maclab_kernels.cuh -- device code of the MacLABSWE step (Zhou,
// arXiv:1902.02999, Section 3) for sm_103a.
//
// Storage: structure of arrays, row pitch `pitch` (a multiple of 64 nodes):
//   eta = h - D (perturbation about still water), u, v   [two copies, ping-pong]
//   D   = h_ref - z_b (still-water depth), in the state precision
//   type: uint8, bits 0-2 node kind, bit 3 = "general links" (some link of
//         the node bounces back, so the interior fast path does not apply)
//
// Perturbation form of Eqs. Mac.lb.6 / Mac.lb.7.  With G6 = g/(6e^2),
// K6 = 1/(6e^2), KF = dt/(6e), lambda_a = 1 (axis) or 1/4 (diagonal),
// C_a = lambda_a / 3, and for a source node y
//     a'(y)  = h (G6 eta - K6 |u|^2)            (f^eq difference, minus G6 eta D)
//     q'(y)  = h u / (3e) + KF F                (first moment plus source force)
//     s(y)   = (h u^2/(2e^2), h v^2/(2e^2), h u v / e^2)
//     o_a(y) = lambda_a [a' + c_a.q' + c_ax^2 s_xx + c_ay^2 s_yy + c_ax c_ay s_xy]
// the still-water part of f^eq_a(y) plus the still-water bed term of each
// link is lambda_a g D(x)^2/(6e^2), independent of y, so it cancels against
// the still-water part of h(x) exactly (lake at rest is exact in any
// precision).  What remains for an interior node x with eight usable links:
//     eta'  = eta - h (5 G6 eta + 4 K6 |u|^2)   (a = 0 term plus the receiver-only
//                                                bed part sum_a lambda_a G6 eta_x D_x)
//             + sum_a o_a(x - c_a)
//             + sum_a lambda_a [G6 D_x eta_y - G6 eta_x D_y]              (bed, cross part)
//     h u'  = e sum_a c_a [o_a(y) + lambda_a (G6 D_x eta_y - G6 eta_x D_y)] + dt F(x) / 2
// where the bed term of each link is -(g/e^2) C_a hbar [z_b(x) - z_b(y)]
// with hbar = (h(x) + h(y))/2 (Eq. h-bar at the old level) and z_b = h_ref - D,
// and the centred force of Eq. force-CS is split into its source half (in
// q') and its receiver half (sum_a lambda_a KF c_a.F(x) = 0 and
// e sum_a lambda_a KF c_a (c_a.F(x)) = dt F(x) / 2).
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda.h>
#include <cuda_runtime.h>

namespace maclab {

enum : uint8_t {
    K_SOLID = 0, K_FLUID = 1, K_NOSLIP = 2, K_DIR_H = 3, K_DIR_Q = 4, K_DIR_HU = 5,
    KIND_MASK = 7, GENERAL_BIT = 8
};
enum : int { EDGE_BB = 0, EDGE_SPEC = 1, EDGE_PER = 2 };

// Constants of one handle, in the state precision T.
template <typename T>
struct Coef {
    T e;     // particle speed (Eq. mlb-viscosity)
    T G6;    // g / (6 e^2)
    T K6;    // 1 / (6 e^2)
    T k3;    // 1 / (3 e)
    T k2;    // 1 / (2 e^2)
    T k1;    // 1 / e^2
    T KF;    // dt / (6 e)
    T hdt;   // dt / 2
    T wfx;   // tau_w,x / rho_w  (Eq. wind_u-stress)
    T wfy;
    T Cb;    // C_b (Eq. bed-stress)
    T Om;    // Omega (Eq. SWE-force)
    T nz;    // -0.0, read at run time (see Op2::mul)
};

template <typename T>
struct Fields {
    const T* eta;
    const T* u;
    const T* v;
    const T* D;
    const uint8_t* type;
    T* eta1;
    T* u1;
    T* v1;
    int nx, ny, pitch;
    int idx32;    // 1 when pitch * ny < 2^31: node offsets fit in an int
    int edge[4];  // W, E, S, N
    Coef<T> c;
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// ---------------------------------------------------------------------------
// Raw node values and the per-source quantities of the fast path.
template <typename T>
struct Raw {
    T eta, u, v, D;
    uint8_t flip;  // bit 0: mirrored in x, bit 1: mirrored in y (specular ghost)
};

template <typename T>
struct Src {
    T eta, D;
    T o1, o2, o3, o4, o5, o6, o7, o8;
    T ownh;        // eta - h (5 G6 eta + 4 K6 |u|^2)
    T hFx, hFy;    // dt F / 2
};

template <typename T>
__device__ __forceinline__ T my_sqrt(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ float my_sqrt<float>(float x) { return sqrtf(x); }

// Correctly rounded operations that the compiler never contracts or
// reorders: the fast path spells out every multiply-add, so a node's result
// does not depend on which inlined copy of the code computed it (and hence
// not on the strip height).
template <typename T> struct Op;
template <> struct Op<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    // hardware approximations (about 1 ulp), ample for the FP32 path
    static __device__ __forceinline__ float rcp(float a)
    {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
    static __device__ __forceinline__ float sqrt(float a)
    {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
        return r;
    }
};
template <> struct Op<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
    static __device__ __forceinline__ double sqrt(double a) { return ::sqrt(a); }
};

// Paired FP32 arithmetic on sm_100-class GPUs: one instruction applies the
// same operation to two lanes (.x, .y), each rounded to nearest as the
// scalar Op<float> operation would be, so a node's result is the same
// whether its arithmetic ran paired or alone.
struct Op2 {
    // The lanes travel as two f32 registers and are packed inside the asm,
    // so no float2 is reinterpreted as an integer in C++.
    static __device__ __forceinline__ float2 add(float2 a, float2 c)
    {
        float2 d;
        asm("{\n .reg .b64 a, c, d;\n mov.b64 a, {%2, %3};\n mov.b64 c, {%4, %5};\n"
            " add.rn.f32x2 d, a, c;\n mov.b64 {%0, %1}, d;\n}\n"
            : "=f"(d.x), "=f"(d.y)
            : "f"(a.x), "f"(a.y), "f"(c.x), "f"(c.y));
        return d;
    }
    static __device__ __forceinline__ float2 sub(float2 a, float2 c)
    {
        float2 d;
        asm("{\n .reg .b64 a, c, d;\n mov.b64 a, {%2, %3};\n mov.b64 c, {%4, %5};\n"
            " sub.rn.f32x2 d, a, c;\n mov.b64 {%0, %1}, d;\n}\n"
            : "=f"(d.x), "=f"(d.y)
            : "f"(a.x), "f"(a.y), "f"(c.x), "f"(c.y));
        return d;
    }
    // a * c as fma(a, c, z) with z = -0.0 from the kernel's parameters: the
    // same rounding as a plain multiply (signed zeros included), but the
    // compiler cannot fuse it into a following add, which it does for a
    // paired multiply even when both carry an explicit rounding mode.
    static __device__ __forceinline__ float2 mul(float2 a, float2 c, float2 z) { return fma(a, c, z); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 c, float2 e)
    {
        float2 d;
        asm("{\n .reg .b64 a, c, e, d;\n mov.b64 a, {%2, %3};\n mov.b64 c, {%4, %5};\n mov.b64 e, {%6, %7};\n"
            " fma.rn.f32x2 d, a, c, e;\n mov.b64 {%0, %1}, d;\n}\n"
            : "=f"(d.x), "=f"(d.y)
            : "f"(a.x), "f"(a.y), "f"(c.x), "f"(c.y), "f"(e.x), "f"(e.y));
        return d;
    }
};
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }

// Which force terms of Eq. SWE-force are present (compile-time variants).
enum : int { F_WIND = 1, F_FRICTION = 2, F_CORIOLIS = 4 };

// Source-side quantities of one node (see the header comment).
template <typename T, int FM>
__device__ __forceinline__ void derive(const Coef<T>& c, const Raw<T>& r, Src<T>& s)
{
    using O = Op<T>;
    T u = r.u, v = r.v, wfx = c.wfx, wfy = c.wfy, Om = c.Om;
    if (r.flip) {  // specular ghost: normal components reversed, rotation sense too
        if (r.flip & 1) { u = -u; wfx = -wfx; }
        if (r.flip & 2) { v = -v; wfy = -wfy; }
        if ((r.flip & 3) != 3) Om = -Om;
    }
    const T eta = r.eta, D = r.D;
    const T h = O::add(D, eta);
    const T uu = O::fma(u, u, O::mul(v, v));
    const T ge = O::mul(c.G6, eta);
    const T ku = O::mul(c.K6, uu);
    const T ap = O::mul(h, O::sub(ge, ku));
    s.ownh = O::fma(-h, O::fma(T(5), ge, O::mul(T(4), ku)), eta);
    // F = tau_w / rho - C_b u |u| + Omega h (v, -u)
    T Fx = (FM & F_WIND) ? wfx : T(0), Fy = (FM & F_WIND) ? wfy : T(0);
    if (FM & F_CORIOLIS) {
        const T omh = O::mul(Om, h);
        Fx = O::fma(omh, v, Fx);
        Fy = O::fma(-omh, u, Fy);
    }
    if (FM & F_FRICTION) {
        const T cbs = O::mul(c.Cb, O::sqrt(uu));
        Fx = O::fma(-cbs, u, Fx);
        Fy = O::fma(-cbs, v, Fy);
    }
    const T hu = O::mul(h, u), hv = O::mul(h, v);
    T qx = O::mul(hu, c.k3), qy = O::mul(hv, c.k3);
    if (FM) {
        s.hFx = O::mul(c.hdt, Fx);
        s.hFy = O::mul(c.hdt, Fy);
        qx = O::fma(c.KF, Fx, qx);
        qy = O::fma(c.KF, Fy, qy);
    } else {
        s.hFx = T(0);
        s.hFy = T(0);
    }
    const T sxx = O::mul(O::mul(hu, u), c.k2);
    const T syy = O::mul(O::mul(hv, v), c.k2);
    const T sxy = O::mul(O::mul(hu, v), c.k1);
    const T ax = O::add(ap, sxx), ay = O::add(ap, syy);
    s.o1 = O::add(ax, qx);
    s.o5 = O::sub(ax, qx);
    s.o3 = O::add(ay, qy);
    s.o7 = O::sub(ay, qy);
    const T d = O::add(ax, syy);
    const T dp = O::mul(T(0.25), O::add(d, sxy)), dm = O::mul(T(0.25), O::sub(d, sxy));
    const T s4 = O::mul(T(0.25), O::add(qx, qy)), t4 = O::mul(T(0.25), O::sub(qx, qy));
    s.o2 = O::add(dp, s4);
    s.o6 = O::sub(dp, s4);
    s.o8 = O::add(dm, t4);
    s.o4 = O::sub(dm, t4);
    s.eta = eta;
    s.D = D;
}

// Source quantities of two nodes at once (FP32): the operations of derive,
// paired.  Negated products are formed with negated constants, which
// rounds to the same value as negating the product.
struct Src2 {
    float2 eta, D;
    float2 o1, o2, o3, o4, o5, o6, o7, o8;
    float2 ownh;
    float2 hFx, hFy;
};

__device__ __forceinline__ void flip_lane(uint8_t fl, float& u, float& v, float& wfx, float& wfy, float& Om)
{
    if (fl & 1) { u = -u; wfx = -wfx; }
    if (fl & 2) { v = -v; wfy = -wfy; }
    if (fl && (fl & 3) != 3) Om = -Om;
}

// The FP32 coefficients as lane pairs (both lanes equal), the operand form
// of the paired instructions; a kernel can take them ready-made in its
// parameters (one 8-byte constant load each) or form them from Coef.
struct Coef2 {
    float2 e, G6, nG6, K6, k3, k2, k1, KF, hdt, nCb, wfx, wfy, Om, nz;
};
__host__ __device__ inline Coef2 coef2_of(const Coef<float>& c)
{
    const auto sp = [](float a) { return make_float2(a, a); };
    return Coef2{sp(c.e), sp(c.G6), sp(-c.G6), sp(c.K6), sp(c.k3), sp(c.k2), sp(c.k1), sp(c.KF), sp(c.hdt),
                 sp(-c.Cb), sp(c.wfx), sp(c.wfy), sp(c.Om), sp(c.nz)};
}

template <int FM>
__device__ __forceinline__ void derive2(const Coef2& c, const Raw<float>& r0, const Raw<float>& r1, Src2& s)
{
    using P = Op2;
    using O = Op<float>;
    const float2 z = c.nz;
    float2 u = make_float2(r0.u, r1.u), v = make_float2(r0.v, r1.v);
    float2 wfx = c.wfx, wfy = c.wfy, Om = c.Om;
    if (r0.flip | r1.flip) {  // specular ghosts: normal components reversed, rotation sense too
        flip_lane(r0.flip, u.x, v.x, wfx.x, wfy.x, Om.x);
        flip_lane(r1.flip, u.y, v.y, wfx.y, wfy.y, Om.y);
    }
    const float2 eta = make_float2(r0.eta, r1.eta), D = make_float2(r0.D, r1.D);
    const float2 h = P::add(D, eta);
    const float2 uu = P::fma(u, u, P::mul(v, v, z));
    const float2 ge = P::mul(c.G6, eta, z);
    const float2 ku = P::mul(c.K6, uu, z);
    const float2 ap = P::mul(h, P::sub(ge, ku), z);
    // eta - h (5 ge + 4 ku)
    s.ownh = P::fma(h, P::fma(splat(-5.f), ge, P::mul(splat(-4.f), ku, z)), eta);
    float2 Fx = (FM & F_WIND) ? wfx : splat(0.f), Fy = (FM & F_WIND) ? wfy : splat(0.f);
    if (FM & F_CORIOLIS) {
        const float2 omh = P::mul(Om, h, z);
        const float2 nomh = P::mul(make_float2(-Om.x, -Om.y), h, z);
        Fx = P::fma(omh, v, Fx);
        Fy = P::fma(nomh, u, Fy);
    }
    if (FM & F_FRICTION) {
        const float2 ncbs = P::mul(c.nCb, make_float2(O::sqrt(uu.x), O::sqrt(uu.y)), z);
        Fx = P::fma(ncbs, u, Fx);
        Fy = P::fma(ncbs, v, Fy);
    }
    const float2 hu = P::mul(h, u, z), hv = P::mul(h, v, z);
    float2 qx = P::mul(hu, c.k3, z), qy = P::mul(hv, c.k3, z);
    if (FM) {
        s.hFx = P::mul(c.hdt, Fx, z);
        s.hFy = P::mul(c.hdt, Fy, z);
        qx = P::fma(c.KF, Fx, qx);
        qy = P::fma(c.KF, Fy, qy);
    } else {
        s.hFx = splat(0.f);
        s.hFy = splat(0.f);
    }
    const float2 sxx = P::mul(P::mul(hu, u, z), c.k2, z);
    const float2 syy = P::mul(P::mul(hv, v, z), c.k2, z);
    const float2 sxy = P::mul(P::mul(hu, v, z), c.k1, z);
    const float2 ax = P::add(ap, sxx), ay = P::add(ap, syy);
    s.o1 = P::add(ax, qx);
    s.o5 = P::sub(ax, qx);
    s.o3 = P::add(ay, qy);
    s.o7 = P::sub(ay, qy);
    const float2 d = P::add(ax, syy);
    const float2 q4 = splat(0.25f);
    const float2 dp = P::mul(q4, P::add(d, sxy), z), dm = P::mul(q4, P::sub(d, sxy), z);
    const float2 s4 = P::mul(q4, P::add(qx, qy), z), t4 = P::mul(q4, P::sub(qx, qy), z);
    s.o2 = P::add(dp, s4);
    s.o6 = P::sub(dp, s4);
    s.o8 = P::add(dm, t4);
    s.o4 = P::sub(dm, t4);
    s.eta = eta;
    s.D = D;
}

// Map a column / row index outside the grid through the edge kinds.
// Returns the in-grid index, or -1 if it lies behind a bounce-back edge or
// maps outside the grid; sets the mirror flag for specular edges.
__device__ __forceinline__ int resolve_index(int i, int n, int lo_kind, int hi_kind, uint8_t bit,
                                             uint8_t& flip)
{
    if (i >= 0 && i < n) return i;
    int kind = i < 0 ? lo_kind : hi_kind;
    if (kind == EDGE_PER) {
        i %= n;
        return i < 0 ? i + n : i;
    }
    if (kind == EDGE_SPEC) {
        i = i < 0 ? -1 - i : 2 * n - 1 - i;
        flip |= bit;
        return (i >= 0 && i < n) ? i : -1;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Fast-path step kernel.  A warp owns a strip of 32*CPL columns (CPL per
// lane) and `ty` rows; it walks the rows, keeping the source quantities of
// three consecutive rows in registers (y neighbours) and exchanging the edge
// columns of each lane with warp shuffles (x neighbours).  Of the strip's
// local columns 0 .. 32 CPL - 1, the W = 31 CPL columns 1 .. W are written:
// strip cb covers global columns [W cb - CPL, W cb - CPL + 32 CPL) and writes
// [W cb - CPL + 1, W cb - CPL + W].
//
// Input rows are staged through a per-warp ring of STAGES rows in shared
// memory with cp.async: each lane copies its own CPL columns of eta, u, v, D
// and reads back only those, so the ring needs no synchronisation beyond
// cp.async.wait_group, and STAGES - 1 rows per warp are in flight while the
// current row is computed.  The type bytes of a row are loaded when the row
// is consumed and unpacked one row later, when it is the output row.
// Build-time tuning knobs (defaults are the measured best on GB300).
#ifndef MACLAB_F32_CPL
#define MACLAB_F32_CPL 4
#endif
#ifndef MACLAB_F32_STAGES
#define MACLAB_F32_STAGES 5
#endif
#ifndef MACLAB_MIN_BLOCKS
#define MACLAB_MIN_BLOCKS 1
#endif
constexpr int WARPS = 4;  // warps per block
template <typename T> struct Cfg;
template <> struct Cfg<float> { static constexpr int CPL = MACLAB_F32_CPL, STAGES = MACLAB_F32_STAGES; };
template <> struct Cfg<double> { static constexpr int CPL = 2, STAGES = 4; };
template <typename T> __host__ __device__ constexpr int strip_width() { return 31 * Cfg<T>::CPL; }

// elements of T per ring slot: 4 fields of 32 CPL values, plus 32 CPL type
// bytes when CPL == 4 (rounded up to whole elements)
template <typename T> __host__ __device__ constexpr int slot_elems()
{
    return 4 * 32 * Cfg<T>::CPL + (Cfg<T>::CPL == 4 ? (32 * Cfg<T>::CPL + (int)sizeof(T) - 1) / (int)sizeof(T) : 0);
}

template <typename T, int CPL> struct VecT;
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<double, 2> { using type = double2; };
template <int CPL> struct TypeWord;
template <> struct TypeWord<4> { using type = uint32_t; };
template <> struct TypeWord<2> { using type = uint16_t; };

template <typename T>
struct Row {
    Src<T> col[Cfg<T>::CPL + 2];  // [0] left neighbour, [1..CPL] own, [CPL+1] right neighbour
    uint32_t types;               // type bytes of the lane's columns (byte k = column k)
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes_valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes_valid));
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, int bytes_valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(bytes_valid));
}
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, int bytes_valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(bytes_valid));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Per-lane column geometry (fixed for the whole strip).
template <int CPL>
struct LaneCols {
    int xl;             // first column of the lane
    bool inside;        // all CPL columns inside the grid
    int src[CPL];       // resolved column (or -1)
    uint8_t flip[CPL];  // x-mirror flag per column
};

// Edge lanes (a column outside the grid or a wrapped / mirrored row): one
// element at a time, resolved through the edge kinds; zero-filled where the
// source lies behind a wall.  Kept out of line so the interior loop stays small.
template <typename T>
__device__ __noinline__ void fetch_row_edge(const Fields<T>& f, const LaneCols<Cfg<T>::CPL>& lc, int rr,
                                            uint32_t slot_addr)
{
    constexpr int CPL = Cfg<T>::CPL;
    const T* fld[4] = {f.eta, f.u, f.v, f.D};
    constexpr uint32_t FSTRIDE = 32 * CPL * sizeof(T);  // bytes per field in a slot
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const bool ok = rr >= 0 && lc.src[k] >= 0;
        const size_t idx = ok ? (size_t)rr * f.pitch + lc.src[k] : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (sizeof(T) == 4)
                cp_async4(slot_addr + q * FSTRIDE + k * sizeof(T), fld[q] + idx, ok ? 4 : 0);
            else
                cp_async8(slot_addr + q * FSTRIDE + k * sizeof(T), fld[q] + idx, ok ? 8 : 0);
        }
    }
}

// Issue the copies of source row r into a ring slot (one commit group).
// Slot layout: eta, u, v, D (32 CPL elements each), then the type bytes
// (32 CPL bytes) when CPL == 4.
template <typename T>
__device__ __forceinline__ void fetch_row(const Fields<T>& f, const LaneCols<Cfg<T>::CPL>& lc, int r,
                                          uint32_t slot_addr, uint32_t type_addr)
{
    constexpr int CPL = Cfg<T>::CPL;
    uint8_t fy = 0;
    const int rr = resolve_index(r, f.ny, f.edge[2], f.edge[3], 2, fy);
    constexpr uint32_t FSTRIDE = 32 * CPL * sizeof(T);  // bytes per field in a slot
    if (rr >= 0 && lc.inside) {
        const size_t base = (size_t)rr * f.pitch + lc.xl;
        const T* fld[4] = {f.eta, f.u, f.v, f.D};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (CPL * sizeof(T) == 16) cp_async16(slot_addr + q * FSTRIDE, fld[q] + base, 16);
            else cp_async8(slot_addr + q * FSTRIDE, fld[q] + base, 8);
        }
        if (CPL == 4) cp_async4(type_addr, f.type + base, 4);
    } else {
        fetch_row_edge(f, lc, rr, slot_addr);
        if (CPL == 4) {
            // the type word of an edge lane is assembled at consume time
        }
    }
    cp_async_commit();
}

// Read the staged row r back, derive its source quantities and exchange the
// edge columns with the neighbouring lanes.
template <typename T, int FM>
__device__ __forceinline__ void consume_row(const Fields<T>& f, const LaneCols<Cfg<T>::CPL>& lc, int r,
                                            const T* slot, int lane, Row<T>& row)
{
    constexpr int CPL = Cfg<T>::CPL;
    constexpr int FE = 32 * CPL;  // elements per field in a slot
    uint8_t fy = 0;
    const int rr = resolve_index(r, f.ny, f.edge[2], f.edge[3], 2, fy);
    using V = typename VecT<T, CPL>::type;
    const V* sp = reinterpret_cast<const V*>(slot + CPL * lane);
    const V e4 = sp[0], u4 = sp[FE / CPL], v4 = sp[2 * FE / CPL], d4 = sp[3 * FE / CPL];
    const T* e = reinterpret_cast<const T*>(&e4);
    const T* u = reinterpret_cast<const T*>(&u4);
    const T* v = reinterpret_cast<const T*>(&v4);
    const T* d = reinterpret_cast<const T*>(&d4);
    if (rr >= 0 && lc.inside) {
        if (CPL == 4)
            row.types = *reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint8_t*>(slot + 4 * FE) + CPL * lane);
        else
            row.types = *reinterpret_cast<const typename TypeWord<CPL>::type*>(f.type + (size_t)rr * f.pitch + lc.xl);
    } else {
        uint32_t t = 0;
#pragma unroll
        for (int k = 0; k < CPL; ++k)
            if (rr >= 0 && lc.src[k] >= 0) t |= (uint32_t)f.type[(size_t)rr * f.pitch + lc.src[k]] << (8 * k);
        row.types = t;
    }
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const Raw<T> raw = {e[k], u[k], v[k], d[k], (uint8_t)(fy | lc.flip[k])};
        derive<T, FM>(f.c, raw, row.col[k + 1]);
    }
    const unsigned full = 0xffffffffu;
    // left neighbour of column 1 = last column of lane-1 (it sends o1, o2, o8)
    Src<T>& L = row.col[0];
    const Src<T>& sl = row.col[CPL];
    L.o1 = __shfl_up_sync(full, sl.o1, 1);
    L.o2 = __shfl_up_sync(full, sl.o2, 1);
    L.o8 = __shfl_up_sync(full, sl.o8, 1);
    L.eta = __shfl_up_sync(full, sl.eta, 1);
    L.D = __shfl_up_sync(full, sl.D, 1);
    // right neighbour of column CPL = first column of lane+1 (it sends o5, o4, o6)
    Src<T>& R = row.col[CPL + 1];
    const Src<T>& sr = row.col[1];
    R.o5 = __shfl_down_sync(full, sr.o5, 1);
    R.o4 = __shfl_down_sync(full, sr.o4, 1);
    R.o6 = __shfl_down_sync(full, sr.o6, 1);
    R.eta = __shfl_down_sync(full, sr.eta, 1);
    R.D = __shfl_down_sync(full, sr.D, 1);
}

// Interior update of output row j from source rows m = j-1, c = j, p = j+1.
template <typename T>
__device__ __forceinline__ void emit_row(const Fields<T>& f, int j, int xl, int lane,
                                         const Row<T>& m, const Row<T>& c, const Row<T>& p)
{
    constexpr int CPL = Cfg<T>::CPL;
    constexpr int W = strip_width<T>();
    const Coef<T>& K = f.c;
    using O = Op<T>;
    T oe[CPL], ou[CPL], ov[CPL];
    unsigned okmask = 0;
#pragma unroll
    for (int k = 1; k <= CPL; ++k) {
        const int loc = CPL * lane + k - 1;  // local column in the strip
        const int x = xl + k - 1;
        const uint8_t ty = (uint8_t)(c.types >> (8 * (k - 1)));
        const bool ok = loc >= 1 && loc <= W && x >= 0 && x < f.nx && (ty & KIND_MASK) != K_SOLID &&
                        !(ty & GENERAL_BIT);
        okmask |= (ok ? 1u : 0u) << (k - 1);
        const Src<T>& mL = m.col[k - 1]; const Src<T>& mC = m.col[k]; const Src<T>& mR = m.col[k + 1];
        const Src<T>& cL = c.col[k - 1]; const Src<T>& cC = c.col[k]; const Src<T>& cR = c.col[k + 1];
        const Src<T>& pL = p.col[k - 1]; const Src<T>& pC = p.col[k]; const Src<T>& pR = p.col[k + 1];
        // streamed equilibria
        const T OL = O::add(O::add(cL.o1, mL.o2), pL.o8);
        const T OR = O::add(O::add(cR.o5, mR.o4), pR.o6);
        const T Sh = O::add(O::add(OL, OR), O::add(mC.o3, pC.o7));
        const T Sx = O::sub(OL, OR);
        const T Sy = O::sub(O::add(O::add(mL.o2, mR.o4), mC.o3), O::add(O::add(pL.o8, pR.o6), pC.o7));
        // lambda-weighted stencils of eta and D: sum, x-moment, y-moment
        const T q = T(0.25);
        const T MLe = O::fma(q, O::add(mL.eta, pL.eta), cL.eta);
        const T MRe = O::fma(q, O::add(mR.eta, pR.eta), cR.eta);
        const T MLd = O::fma(q, O::add(mL.D, pL.D), cL.D);
        const T MRd = O::fma(q, O::add(mR.D, pR.D), cR.D);
        const T Se = O::add(O::add(MLe, MRe), O::add(mC.eta, pC.eta));
        const T Sd = O::add(O::add(MLd, MRd), O::add(mC.D, pC.D));
        const T Xe = O::sub(MLe, MRe), Xd = O::sub(MLd, MRd);
        const T Ye = O::fma(q, O::sub(O::add(mL.eta, mR.eta), O::add(pL.eta, pR.eta)), O::sub(mC.eta, pC.eta));
        const T Yd = O::fma(q, O::sub(O::add(mL.D, mR.D), O::add(pL.D, pR.D)), O::sub(mC.D, pC.D));
        const T etax = cC.eta, Dx = cC.D;
        const T A = O::mul(K.G6, Dx), B = O::mul(K.G6, etax);
        // ownh already holds the receiver-only bed part 5 G6 eta_x D_x
        const T eta1 = O::add(O::add(cC.ownh, Sh), O::fma(A, Se, O::mul(-B, Sd)));
        const T hu1 = O::fma(K.e, O::add(Sx, O::fma(A, Xe, O::mul(-B, Xd))), cC.hFx);
        const T hv1 = O::fma(K.e, O::add(Sy, O::fma(A, Ye, O::mul(-B, Yd))), cC.hFy);
        const T inv = O::rcp(O::add(Dx, eta1));
        const bool noslip = (ty & KIND_MASK) == K_NOSLIP;
        oe[k - 1] = eta1;
        ou[k - 1] = noslip ? T(0) : O::mul(hu1, inv);
        ov[k - 1] = noslip ? T(0) : O::mul(hv1, inv);
    }
    if (j >= f.ny || okmask == 0) return;
    const size_t row0 = (size_t)j * f.pitch;
    using V = typename VecT<T, CPL>::type;
    if (okmask == (1u << CPL) - 1) {
        *reinterpret_cast<V*>(f.eta1 + row0 + xl) = *reinterpret_cast<const V*>(oe);
        *reinterpret_cast<V*>(f.u1 + row0 + xl) = *reinterpret_cast<const V*>(ou);
        *reinterpret_cast<V*>(f.v1 + row0 + xl) = *reinterpret_cast<const V*>(ov);
    } else {
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            if (okmask & (1u << k)) {
                f.eta1[row0 + xl + k] = oe[k];
                f.u1[row0 + xl + k] = ou[k];
                f.v1[row0 + xl + k] = ov[k];
            }
        }
    }
}

// One strip: rows [j0, j1) of column strip cb.
template <typename T, int FM>
__device__ __forceinline__ void step_strip(const Fields<T>& f, int cb, int j0, int j1, int lane,
                                           T (*my)[slot_elems<T>()])
{
    constexpr int CPL = Cfg<T>::CPL, S = Cfg<T>::STAGES;
    constexpr int SLOT = slot_elems<T>();  // elements of T per ring slot
    LaneCols<CPL> lc;
    lc.xl = strip_width<T>() * cb - CPL + CPL * lane;
    lc.inside = lc.xl >= 0 && lc.xl + CPL <= f.nx;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        lc.flip[k] = 0;
        lc.src[k] = resolve_index(lc.xl + k, f.nx, f.edge[0], f.edge[1], 1, lc.flip[k]);
    }
    const int nrows = j1 - j0 + 2;  // source rows j0-1 .. j1
    const uint32_t ring_addr = (uint32_t)__cvta_generic_to_shared(&my[0][0]) + lane * CPL * sizeof(T);
    const uint32_t type_off = 4 * 32 * CPL * sizeof(T) - lane * CPL * sizeof(T) + lane * CPL;
    constexpr uint32_t SLOT_BYTES = SLOT * sizeof(T);
    // prologue: S-1 rows in flight
#pragma unroll
    for (int q = 0; q < S - 1; ++q) {
        if (q < nrows) fetch_row(f, lc, j0 - 1 + q, ring_addr + q * SLOT_BYTES, ring_addr + q * SLOT_BYTES + type_off);
        else cp_async_commit();
    }
    int slot_c = 0;          // ring slot of the next row to consume
    int slot_f = S - 1;      // ring slot of the next row to fetch
    int q = 0;               // index of the next row to consume
    // consume row q after issuing row q + S - 1
    auto advance = [&](Row<T>& dst) {
        if (q + S - 1 < nrows)
            fetch_row(f, lc, j0 - 1 + q + S - 1, ring_addr + slot_f * SLOT_BYTES,
                      ring_addr + slot_f * SLOT_BYTES + type_off);
        else cp_async_commit();
        cp_async_wait<S - 1>();
        consume_row<T, FM>(f, lc, j0 - 1 + q, &my[slot_c][0], lane, dst);
        slot_c = slot_c == S - 1 ? 0 : slot_c + 1;
        slot_f = slot_f == S - 1 ? 0 : slot_f + 1;
        ++q;
    };
    Row<T> A, B, C;
    advance(A);
    advance(B);
    // rows rotate A -> B -> C so that no register copies of Row are needed
    for (int j = j0;; j += 3) {
        advance(C);
        emit_row(f, j, lc.xl, lane, A, B, C);
        if (j + 1 >= j1) break;
        advance(A);
        emit_row(f, j + 1, lc.xl, lane, B, C, A);
        if (j + 2 >= j1) break;
        advance(B);
        emit_row(f, j + 2, lc.xl, lane, C, A, B);
        if (j + 3 >= j1) break;
    }
    cp_async_wait<0>();
}

// Warps take strips (cb, rb) in turn; with a grid smaller than the strip
// count each warp walks several strips (persistent launch).
template <typename T, int FM>
__global__ void __launch_bounds__(32 * WARPS, MACLAB_MIN_BLOCKS)
step_fast_kernel(const Fields<T> f, int ncb, int nrb, int ty)
{
    constexpr int S = Cfg<T>::STAGES;
    constexpr int SLOT = slot_elems<T>();
    __shared__ __align__(16) T ring[WARPS][S][SLOT];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = (int)(gridDim.x * (blockDim.x >> 5));
    const int nstrips = ncb * nrb;
    for (int strip = (int)(blockIdx.x * (blockDim.x >> 5)) + wib; strip < nstrips; strip += nwarps) {
        const int cb = strip % ncb, rb = strip / ncb;
        const int j0 = rb * ty;
        step_strip<T, FM>(f, cb, j0, min(f.ny, j0 + ty), lane, ring[wib]);
    }
}

// ---------------------------------------------------------------------------
// General-link kernel: nodes with at least one bounce-back link (next to a
// solid node or a bounce-back edge).  Each link is resolved as in the
// paper's boundary rules: a solid or walled-off source bounces back
// (f^eq of the opposite direction at the node itself, no bed or force
// term); a specular source is the mirror image; a periodic source wraps.
__constant__ int c_cx[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
__constant__ int c_cy[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};

template <typename T>
struct NodeQ {  // per-node quantities for the general path
    T eta, D, h, u, v, uu, Fx, Fy;
};

template <typename T>
__device__ __forceinline__ NodeQ<T> node_q(const Fields<T>& f, size_t idx, uint8_t flip)
{
    using O = Op<T>;
    const Coef<T>& c = f.c;
    NodeQ<T> n;
    n.eta = f.eta[idx];
    n.D = f.D[idx];
    n.u = f.u[idx];
    n.v = f.v[idx];
    T wfx = c.wfx, wfy = c.wfy, Om = c.Om;
    if (flip & 1) { n.u = -n.u; wfx = -wfx; }
    if (flip & 2) { n.v = -n.v; wfy = -wfy; }
    if ((flip & 3) == 1 || (flip & 3) == 2) Om = -Om;
    n.h = O::add(n.D, n.eta);
    n.uu = O::fma(n.u, n.u, O::mul(n.v, n.v));
    const T sp = Op<T>::sqrt(n.uu);
    const T cbs = O::mul(c.Cb, sp), omh = O::mul(Om, n.h);
    n.Fx = O::fma(-cbs, n.u, O::fma(omh, n.v, wfx));
    n.Fy = O::fma(-cbs, n.v, O::fma(-omh, n.u, wfy));
    return n;
}

// f^eq_a(h,u) - f^eq_a(D,0) for direction a != 0 with lattice vector (cx, cy)
template <typename T>
__device__ __forceinline__ T feq_diff(const Coef<T>& c, const NodeQ<T>& n, int cx, int cy)
{
    using O = Op<T>;
    const T lam = (cx != 0 && cy != 0) ? T(0.25) : T(1);
    const T cu = O::fma(T(cx), n.u, O::mul(T(cy), n.v));
    const T hcu = O::mul(n.h, cu);
    T acc = O::mul(O::mul(c.G6, n.eta), O::fma(T(2), n.D, n.eta));
    acc = O::fma(hcu, c.k3, acc);
    acc = O::fma(O::mul(hcu, cu), c.k2, acc);
    acc = O::fma(-c.K6, O::mul(n.h, n.uu), acc);
    return O::mul(lam, acc);
}

// Update of one node (i, j) with the links resolved one by one.  Every
// rounding is spelled out, so the result does not depend on which kernel
// the code is inlined into.  NEW: hbar at the new time level (Eq. h-bar as
// written, hbar = (h(x, t + dt) + h(y, t)) / 2): the bed terms are linear in
// the new eta of the node, which is then solved for directly.
template <typename T, bool NEW = false>
__device__ __forceinline__ void general_node(const Fields<T>& f, int i, int j)
{
    using O = Op<T>;
    const size_t xi = (size_t)j * f.pitch + i;
    const Coef<T>& c = f.c;
    const NodeQ<T> X = node_q(f, xi, 0);
    T Sh = O::fma(-O::mul(T(5), O::mul(c.G6, X.eta)), O::fma(T(2), X.D, X.eta), X.eta);
    Sh = O::fma(-O::mul(T(4), c.K6), O::mul(X.h, X.uu), Sh);
    T Sx = T(0), Sy = T(0);
    T Q = T(0), Qx = T(0), Qy = T(0);  // new level: sum of lambda G6 (D_x - D_y), weighted by 1, c_x, c_y
#pragma unroll 1
    for (int a = 1; a < 9; ++a) {
        const int cx = c_cx[a], cy = c_cy[a];
        const T lam = (a & 1) ? T(1) : T(0.25);
        uint8_t flip = 0;
        const int si = resolve_index(i - cx, f.nx, f.edge[0], f.edge[1], 1, flip);
        const int sj = resolve_index(j - cy, f.ny, f.edge[2], f.edge[3], 2, flip);
        bool bounce = si < 0 || sj < 0;
        size_t s = 0;
        if (!bounce) {
            s = (size_t)sj * f.pitch + si;
            bounce = (f.type[s] & KIND_MASK) == K_SOLID;
        }
        T w;
        if (bounce) {
            w = feq_diff(c, X, -cx, -cy);
        } else {
            const NodeQ<T> Y = node_q(f, s, flip);  // the mirrored node when flip != 0
            T bed;
            if (NEW) {
                const T q = O::mul(O::mul(lam, c.G6), O::sub(X.D, Y.D));
                bed = O::mul(q, Y.eta);  // the source half; the node's half waits for its new eta
                Q = O::add(Q, q);
                Qx = O::fma(T(cx), q, Qx);
                Qy = O::fma(T(cy), q, Qy);
            } else {
                bed = O::mul(O::mul(lam, c.G6), O::mul(O::add(X.eta, Y.eta), O::sub(X.D, Y.D)));
            }
            const T frc = O::mul(O::mul(lam, c.KF),
                                 O::fma(T(cx), O::add(X.Fx, Y.Fx), O::mul(T(cy), O::add(X.Fy, Y.Fy))));
            w = O::add(O::add(feq_diff(c, Y, cx, cy), bed), frc);
        }
        Sh = O::add(Sh, w);
        Sx = O::fma(T(cx), w, Sx);
        Sy = O::fma(T(cy), w, Sy);
    }
    if (NEW) {  // eta1 = Sh + eta1 Q
        Sh = Sh / O::sub(T(1), Q);
        Sx = O::fma(Sh, Qx, Sx);
        Sy = O::fma(Sh, Qy, Sy);
    }
    const T hu1 = O::mul(c.e, Sx), hv1 = O::mul(c.e, Sy);
    const T inv = T(1) / O::add(X.D, Sh);
    T u1 = O::mul(hu1, inv), v1 = O::mul(hv1, inv);
    if ((f.type[xi] & KIND_MASK) == K_NOSLIP) { u1 = T(0); v1 = T(0); }
    f.eta1[xi] = Sh;
    f.u1[xi] = u1;
    f.v1[xi] = v1;
}

template <typename T, bool NEW = false>
__global__ void __launch_bounds__(128) step_general_kernel(const Fields<T> f, const int* __restrict__ list,
                                                           int count)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int node = list[t];
    general_node<T, NEW>(f, node % f.nx, node / f.nx);
}

// ---------------------------------------------------------------------------
// Dirichlet nodes, after every other node holds its new value: prescribed
// quantities take their value at t_{n+1}; the unprescribed one takes the new
// value of the first node inward along the edge normal (zero gradient).
struct DirNode {
    int x, n1;  // storage indices (row * pitch + col) of the node and its inward node
    int meta;   // kind | (edge << 4)
};
struct DirValues {
    double h[4], qx[4], qy[4];  // prescribed values at t_{n+1} per edge
};

template <typename T>
__device__ __forceinline__ void dirichlet_node(T* eta, T* u, T* v, const T* D, const double* D64, const DirNode d,
                                               const DirValues& bv)
{
    const int kind = d.meta & 15, ed = d.meta >> 4;
    if (kind == K_DIR_H) {
        eta[d.x] = (T)(bv.h[ed] - D64[d.x]);
        u[d.x] = u[d.n1];
        v[d.x] = v[d.n1];
        return;
    }
    const double h = kind == K_DIR_Q ? (double)D[d.n1] + (double)eta[d.n1] : bv.h[ed];
    eta[d.x] = (T)(h - D64[d.x]);
    u[d.x] = (T)(bv.qx[ed] / h);
    v[d.x] = (T)(bv.qy[ed] / h);
}

template <typename T>
__global__ void dirichlet_kernel(T* __restrict__ eta, T* __restrict__ u, T* __restrict__ v,
                                 const T* __restrict__ D, const double* __restrict__ D64,
                                 const DirNode* __restrict__ list, int count, const DirValues bv)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    dirichlet_node(eta, u, v, D, D64, list[t], bv);
}

// ---------------------------------------------------------------------------
// Tile step kernel (the default).  A 256-thread block updates a tile of
// TX x TY = 64 x 16 nodes:
//   A. every thread loads node pairs of the tile plus its one-node halo
//      (68 x 18 nodes), derives their source quantities and writes the eight
//      outgoing values and (eta, D) to shared memory; the pairs it updates
//      keep their own term, dt F / 2 and types in registers;
//   B. after a barrier every thread gathers, for each of its 2 x 2 nodes,
//      the eight incoming values and the eta / D stencils and writes
//      eta, u, v (nodes with a bounce-back link are left to
//      step_general_kernel);
//   C. when every Dirichlet node's inward node lies in the same tile and
//      has no bounce-back link, the tile's Dirichlet nodes are set from the
//      new values after a second barrier.
// Thread (tx, ty) of 32 x 8 owns the node pairs at tile columns 2 + 2 tx,
// 3 + 2 tx of tile rows 1 + 2 ty and 2 + 2 ty.  Tiles whose reads and
// writes all lie inside the grid (every tile but the outermost ring) load
// without edge rules or bounds tests, with 32-bit node offsets.
namespace tile {
#ifndef MACLAB_TILE_TY
#define MACLAB_TILE_TY 16
#endif
constexpr int TX = 64, TY = MACLAB_TILE_TY;  // nodes updated per tile
constexpr int THREADS = 16 * TY;           // 32 x TY / 2
constexpr int PC = TX / 2 + 2;             // 34 node pairs per tile row (with halo)
constexpr int IR = TY + 2;                 // 18 tile rows (with halo)
constexpr int IW = 2 * PC;                 // 68 tile columns: global x0 - 2 .. x0 + 65
constexpr int HALO_PAIRS = 2 * IR + 2 * (PC - 2);  // 100
template <typename T, int ROWS = IR>
struct Derived {
    T o_[8][ROWS][IW];                     // outgoing values o_1 .. o_8
    __device__ __forceinline__ T& o(int d, int r, int c) { return o_[d][r][c]; }
    __device__ __forceinline__ const T& o(int d, int r, int c) const { return o_[d][r][c]; }
    // (eta, D), even and odd tile columns apart: a warp reading column
    // 2 tx + k (k fixed) then touches consecutive 8-byte words
    typename Vec2<T>::type ed_[2][ROWS][IW / 2];
    __device__ __forceinline__ typename Vec2<T>::type& ed(int r, int c) { return ed_[c & 1][r][c >> 1]; }
    __device__ __forceinline__ const typename Vec2<T>::type& ed(int r, int c) const { return ed_[c & 1][r][c >> 1]; }
};
#ifndef MACLAB_TILE_MINB
#define MACLAB_TILE_MINB 4
#endif
template <typename T> struct MinBlocks { static constexpr int value = MACLAB_TILE_MINB; };
template <> struct MinBlocks<double> { static constexpr int value = 2; };
// the batch kernel carries per-instance state; at four blocks per SM a few
// bytes of it spill, which costs less than the fourth block gains (0.565 ->
// 0.521 ms per step of 512 instances)
#ifndef MACLAB_BATCH_MINB
#define MACLAB_BATCH_MINB 4
#endif
template <typename T> struct BatchMinBlocks { static constexpr int value = MACLAB_BATCH_MINB; };
template <> struct BatchMinBlocks<double> { static constexpr int value = 2; };
template <typename T>
__host__ __device__ constexpr size_t smem_bytes() { return sizeof(Derived<T>); }
}  // namespace tile

// Dirichlet nodes handled inside the tile kernel: those of tile t are
// list[start[t] .. start[t + 1]).
struct TileDirichlet {
    const int* start;      // nullptr when the tile kernel does not handle them
    const DirNode* list;
    const double* D64;
    DirValues bv;
    // nodes with a bounce-back link of tile t: glist[gstart[t] .. gstart[t + 1])
    // (j * nx + i), or nullptr when a separate launch updates them
    const int* gstart;
    const int* glist;
};

template <typename T>
__device__ __forceinline__ void load_pair(const Fields<T>& f, int y, int x, Raw<T> (&raw)[2], uint32_t& types)
{
    uint8_t fy = 0;
    const int rr = resolve_index(y, f.ny, f.edge[2], f.edge[3], 2, fy);
    if (rr >= 0 && x >= 0 && x + 2 <= f.nx) {
        const size_t base = (size_t)rr * f.pitch + x;
        using V2 = typename Vec2<T>::type;
        const V2 e2 = *reinterpret_cast<const V2*>(f.eta + base);
        const V2 u2 = *reinterpret_cast<const V2*>(f.u + base);
        const V2 v2 = *reinterpret_cast<const V2*>(f.v + base);
        const V2 d2 = *reinterpret_cast<const V2*>(f.D + base);
        types = *reinterpret_cast<const uint16_t*>(f.type + base);
        raw[0] = Raw<T>{e2.x, u2.x, v2.x, d2.x, fy};
        raw[1] = Raw<T>{e2.y, u2.y, v2.y, d2.y, fy};
        return;
    }
    types = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        uint8_t fl = fy;
        const int cc = resolve_index(x + k, f.nx, f.edge[0], f.edge[1], 1, fl);
        if (rr >= 0 && cc >= 0) {
            const size_t idx = (size_t)rr * f.pitch + cc;
            raw[k] = Raw<T>{f.eta[idx], f.u[idx], f.v[idx], f.D[idx], fl};
            types |= (uint32_t)f.type[idx] << (8 * k);
        } else {
            raw[k] = Raw<T>{T(0), T(0), T(0), T(0), 0};
        }
    }
}

// Phase A of the tile at (x0, y0) reads grid rows y0 - 1 .. y0 + 16 and
// columns x0 - 2 .. x0 + 65 only.
__device__ __forceinline__ bool tile_interior(int nx, int ny, int x0, int y0)
{
    return x0 >= 2 && x0 + tile::TX + 2 <= nx && y0 >= 1 && y0 + tile::TY + 1 <= ny;
}
// A tile whose reads and writes all lie inside the grid (no edge rule, no
// bounds test) and whose offsets fit in 32 bits.
template <typename T>
__device__ __forceinline__ bool tile_inside(const Fields<T>& f, int x0, int y0)
{
    return f.idx32 && tile_interior(f.nx, f.ny, x0, y0);
}

// The pair at node offset `off` of an inside tile.
template <typename T>
__device__ __forceinline__ void load_pair_in(const Fields<T>& f, int off, Raw<T> (&raw)[2], uint32_t& types)
{
    using V2 = typename Vec2<T>::type;
    const V2 e2 = *reinterpret_cast<const V2*>(f.eta + off);
    const V2 u2 = *reinterpret_cast<const V2*>(f.u + off);
    const V2 v2 = *reinterpret_cast<const V2*>(f.v + off);
    const V2 d2 = *reinterpret_cast<const V2*>(f.D + off);
    types = *reinterpret_cast<const uint16_t*>(f.type + off);
    raw[0] = Raw<T>{e2.x, u2.x, v2.x, d2.x, 0};
    raw[1] = Raw<T>{e2.y, u2.y, v2.y, d2.y, 0};
}

template <typename T>
__device__ __forceinline__ void store_pair(tile::Derived<T>& sm, int pr, int lc, const Src<T>& a, const Src<T>& b)
{
    using V2 = typename Vec2<T>::type;
    const T oa[8] = {a.o1, a.o2, a.o3, a.o4, a.o5, a.o6, a.o7, a.o8};
    const T ob[8] = {b.o1, b.o2, b.o3, b.o4, b.o5, b.o6, b.o7, b.o8};
#pragma unroll
    for (int d = 0; d < 8; ++d) *reinterpret_cast<V2*>(&sm.o(d, pr, lc)) = V2{oa[d], ob[d]};
    sm.ed(pr, lc) = V2{a.eta, a.D};
    sm.ed(pr, lc + 1) = V2{b.eta, b.D};
}

// Raw rows of an interior tile staged in shared memory by tensor copies
// (FP32): eta, u, v and D over global columns x0 - 4 .. x0 + 67 (a 16-byte
// aligned start) and the node types over x0 - 16 .. x0 + 79, for tile rows
// y0 - 1 .. y0 + 16.  A tensor copy writes to a 128-byte aligned shared
// address, so each staged field starts on 128 bytes.
namespace tma {
constexpr int SRW = tile::TX + 8;     // 72 staged float columns
constexpr int STW = tile::TX + 32;    // 96 staged type columns
constexpr int FOFF = 2;               // staged float column of tile column 0
constexpr int TOFF = 14;              // staged type column of tile column 0
constexpr int FBOX = tile::IR * SRW;  // floats per staged field (5184 bytes)
constexpr int FSTRIDE = (FBOX * 4 + 127) / 128 * 128 / 4;  // floats between fields (5248 bytes)
struct Stage {
    float f[4][FSTRIDE];              // eta, u, v, D: [IR][SRW] each
    uint8_t type[tile::IR * STW];     // [IR][STW]
};
constexpr uint32_t BYTES = 4u * FBOX * 4u + tile::IR * STW;
constexpr size_t STAGE_OFF = (sizeof(tile::Derived<float>) + 127) / 128 * 128;
constexpr size_t SMEM = 128 + STAGE_OFF + sizeof(Stage);  // 128: room to align the base
}  // namespace tma

// Pair at tile row lr and tile column lc (even) of a staged tile.
__device__ __forceinline__ void staged_pair(const tma::Stage& st, int lr, int lc, Raw<float> (&raw)[2],
                                            uint32_t& types)
{
    const int s = lr * tma::SRW + lc + tma::FOFF;
    const float2 e2 = *reinterpret_cast<const float2*>(&st.f[0][s]);
    const float2 u2 = *reinterpret_cast<const float2*>(&st.f[1][s]);
    const float2 v2 = *reinterpret_cast<const float2*>(&st.f[2][s]);
    const float2 d2 = *reinterpret_cast<const float2*>(&st.f[3][s]);
    types = *reinterpret_cast<const uint16_t*>(&st.type[lr * tma::STW + lc + tma::TOFF]);
    raw[0] = Raw<float>{e2.x, u2.x, v2.x, d2.x, 0};
    raw[1] = Raw<float>{e2.y, u2.y, v2.y, d2.y, 0};
}

// Phase A of a tile: raw values of the thread's own pairs (tile pair
// column 1 + tx, tile rows 1 + 2 tyy + r) and of one halo pair, loaded
// through the edge rules, derived one node at a time and stored to shared
// memory (FP64; FP32 uses the paired tile_phase_a_f32).
template <typename T, int FM>
__device__ __forceinline__ void tile_phase_a(const Fields<T>& f, int x0, int y0, bool inside, tile::Derived<T>& sm,
                                             Src<T> (&own)[2][2], uint32_t (&own_types)[2])
{
    using namespace tile;
    const int tx = threadIdx.x & 31, tyy = threadIdx.x >> 5;
    Raw<T> raw[2][2];
    Raw<T> hraw[2];
    uint32_t htypes;
    int hpr = 0, hpc = 0;
    const bool has_halo = threadIdx.x < HALO_PAIRS;
    if (has_halo) {
        const int h = threadIdx.x;
        if (h < 2 * IR) { hpc = h < IR ? 0 : PC - 1; hpr = h % IR; }
        else { const int u = h - 2 * IR; hpr = u < PC - 2 ? 0 : IR - 1; hpc = 1 + u % (PC - 2); }
    }
    if (inside) {
        const int off = (y0 + 2 * tyy) * f.pitch + x0 + 2 * tx;
        load_pair_in(f, off, raw[0], own_types[0]);
        load_pair_in(f, off + f.pitch, raw[1], own_types[1]);
        if (has_halo) load_pair_in(f, (y0 - 1 + hpr) * f.pitch + x0 - 2 + 2 * hpc, hraw, htypes);
    } else {
#pragma unroll
        for (int r = 0; r < 2; ++r) load_pair(f, y0 + 2 * tyy + r, x0 + 2 * tx, raw[r], own_types[r]);
        if (has_halo) load_pair(f, y0 - 1 + hpr, x0 - 2 + 2 * hpc, hraw, htypes);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        derive<T, FM>(f.c, raw[r][0], own[r][0]);
        derive<T, FM>(f.c, raw[r][1], own[r][1]);
        store_pair(sm, 1 + 2 * tyy + r, 2 + 2 * tx, own[r][0], own[r][1]);
    }
    if (has_halo) {
        Src<T> h0, h1;
        derive<T, FM>(f.c, hraw[0], h0);
        derive<T, FM>(f.c, hraw[1], h1);
        store_pair(sm, hpr, 2 * hpc, h0, h1);
    }
}

// New eta, u, v of a node from its streamed sums (Sh, Sx, Sy: the first
// terms of Eqs. Mac.lb.6 / Mac.lb.7 over the eight incoming outgoing values)
// and the (eta, D) of its eight neighbours (m: row above, c: same row,
// p: row below; L / C / R: column left / same / right), in the perturbation
// form; eta, D, ownh, hFx, hFy are the node's own source quantities.  Every
// kernel that updates fast-path nodes ends in this one function, so their
// results agree bitwise.
template <typename T, typename V2 = typename Vec2<T>::type>
__device__ __forceinline__ void update_tail(const Coef<T>& K, T Sh, T Sx, T Sy, V2 mL, V2 mC, V2 mR, V2 cL, V2 cR,
                                            V2 pL, V2 pC, V2 pR, T eta, T D, T ownh, T hFx, T hFy, bool noslip,
                                            T& oe, T& ou, T& ov)
{
    using O = Op<T>;
    const T q = T(0.25);
    // lambda-weighted stencils of eta (.x) and D (.y): sum, x-moment, y-moment
    T Se, Sd, Xe, Xd, Ye, Yd;
#ifndef MACLAB_SCALAR_STENCIL
    if constexpr (std::is_same<T, float>::value) {
        // eta and D take the same operations: the two lanes of one paired
        // instruction (each lane rounded as the scalar operation)
        using P = Op2;
        const float2 q2 = splat(q);
        const float2 ML = P::fma(q2, P::add(mL, pL), cL), MR = P::fma(q2, P::add(mR, pR), cR);
        const float2 S = P::add(P::add(ML, MR), P::add(mC, pC));
        const float2 X = P::sub(ML, MR);
        const float2 Y = P::fma(q2, P::sub(P::add(mL, mR), P::add(pL, pR)), P::sub(mC, pC));
        Se = S.x, Sd = S.y, Xe = X.x, Xd = X.y, Ye = Y.x, Yd = Y.y;
    } else
#endif
    {
        const T MLe = O::fma(q, O::add(mL.x, pL.x), cL.x);
        const T MRe = O::fma(q, O::add(mR.x, pR.x), cR.x);
        const T MLd = O::fma(q, O::add(mL.y, pL.y), cL.y);
        const T MRd = O::fma(q, O::add(mR.y, pR.y), cR.y);
        Se = O::add(O::add(MLe, MRe), O::add(mC.x, pC.x));
        Sd = O::add(O::add(MLd, MRd), O::add(mC.y, pC.y));
        Xe = O::sub(MLe, MRe), Xd = O::sub(MLd, MRd);
        Ye = O::fma(q, O::sub(O::add(mL.x, mR.x), O::add(pL.x, pR.x)), O::sub(mC.x, pC.x));
        Yd = O::fma(q, O::sub(O::add(mL.y, mR.y), O::add(pL.y, pR.y)), O::sub(mC.y, pC.y));
    }
    const T A = O::mul(K.G6, D), B = O::mul(K.G6, eta);
    // ownh already holds the receiver-only bed part 5 G6 eta_x D_x
    const T eta1 = O::add(O::add(ownh, Sh), O::fma(A, Se, O::mul(-B, Sd)));
    const T hu1 = O::fma(K.e, O::add(Sx, O::fma(A, Xe, O::mul(-B, Xd))), hFx);
    const T hv1 = O::fma(K.e, O::add(Sy, O::fma(A, Ye, O::mul(-B, Yd))), hFy);
    const T inv = O::rcp(O::add(D, eta1));
    oe = eta1;
    ou = noslip ? T(0) : O::mul(hu1, inv);
    ov = noslip ? T(0) : O::mul(hv1, inv);
}

// Streamed sums of the first terms of Eqs. Mac.lb.6 / Mac.lb.7 from the
// eight incoming values, grouped as (left column), (right column), centre:
// a1 = cL_o1 + mL_o2 and a2 = cR_o5 + mR_o4 and sym = mL_o2 + mR_o4 + mC_o3
// take only the node's own row and the row above, so a kernel that walks
// down the rows can form them before the row below exists.
template <typename T>
__device__ __forceinline__ void streamed_sums(T a1, T a2, T sym, T mC_o3, T pL_o8, T pR_o6, T pC_o7, T& Sh, T& Sx,
                                              T& Sy)
{
    using O = Op<T>;
    const T OL = O::add(a1, pL_o8);
    const T OR = O::add(a2, pR_o6);
    Sh = O::add(O::add(OL, OR), O::add(mC_o3, pC_o7));
    Sx = O::sub(OL, OR);
    Sy = O::sub(sym, O::add(O::add(pL_o8, pR_o6), pC_o7));
}

// New eta, u, v of the node at tile row lr, column lc from the derived values
// of its eight neighbours in shared memory (Eqs. Mac.lb.6 / Mac.lb.7 in the
// perturbation form); eta, D, ownh, hFx, hFy are the node's own source
// quantities.
template <typename T, typename DR>
__device__ __forceinline__ void node_update(const DR& sm, int lr, int lc, const Coef<T>& K, T eta, T D, T ownh,
                                            T hFx, T hFy, bool noslip, T& oe, T& ou, T& ov)
{
    using O = Op<T>;
    const T cL_o1 = sm.o(0, lr, lc - 1), mL_o2 = sm.o(1, lr - 1, lc - 1), pL_o8 = sm.o(7, lr + 1, lc - 1);
    const T cR_o5 = sm.o(4, lr, lc + 1), mR_o4 = sm.o(3, lr - 1, lc + 1), pR_o6 = sm.o(5, lr + 1, lc + 1);
    const T mC_o3 = sm.o(2, lr - 1, lc), pC_o7 = sm.o(6, lr + 1, lc);
    T Sh, Sx, Sy;
    streamed_sums<T>(O::add(cL_o1, mL_o2), O::add(cR_o5, mR_o4), O::add(O::add(mL_o2, mR_o4), mC_o3), mC_o3, pL_o8,
                     pR_o6, pC_o7, Sh, Sx, Sy);
    update_tail<T>(K, Sh, Sx, Sy, sm.ed(lr - 1, lc - 1), sm.ed(lr - 1, lc), sm.ed(lr - 1, lc + 1), sm.ed(lr, lc - 1),
                   sm.ed(lr, lc + 1), sm.ed(lr + 1, lc - 1), sm.ed(lr + 1, lc), sm.ed(lr + 1, lc + 1), eta, D, ownh,
                   hFx, hFy, noslip, oe, ou, ov);
}

// Phases B and C of a tile whose phase A is complete and visible; `tile`
// indexes the per-tile Dirichlet ranges.
template <typename T>
__device__ __forceinline__ void tile_phase_bc(const Fields<T>& f, int x0, int y0, bool inside, int tile,
                                              const int* dir_start, const DirNode* dir_list, const double* D64,
                                              const DirValues& bv, const tile::Derived<T>& sm,
                                              const Src<T> (&own)[2][2], const uint32_t (&own_types)[2])
{
    using namespace tile;
    using V2 = typename Vec2<T>::type;
    const int tx = threadIdx.x & 31, tyy = threadIdx.x >> 5;
    const Coef<T>& K = f.c;
    // ---- phase B: nodes (x0 + 2 tx + k, y0 + 2 tyy + r)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int lr = 1 + 2 * tyy + r;    // tile row of the node
        const int y = y0 + 2 * tyy + r;
        T oe[2], ou[2], ov[2];
        unsigned okmask = 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int lc = 2 + 2 * tx + k;  // tile column of the node
            const int x = x0 + 2 * tx + k;
            const uint8_t ty = (uint8_t)(own_types[r] >> (8 * k));
            const bool ok = (inside || (x < f.nx && y < f.ny)) && (ty & KIND_MASK) != K_SOLID && !(ty & GENERAL_BIT);
            okmask |= (ok ? 1u : 0u) << k;
            const Src<T>& me = own[r][k];
            node_update<T>(sm, lr, lc, K, me.eta, me.D, me.ownh, me.hFx, me.hFy,
                           (ty & KIND_MASK) == K_NOSLIP, oe[k], ou[k], ov[k]);
        }
        if (okmask == 0) continue;
        const size_t idx = inside ? (size_t)(y * f.pitch + x0 + 2 * tx) : (size_t)y * f.pitch + x0 + 2 * tx;
        if (okmask == 3u) {
            *reinterpret_cast<V2*>(f.eta1 + idx) = V2{oe[0], oe[1]};
            *reinterpret_cast<V2*>(f.u1 + idx) = V2{ou[0], ou[1]};
            *reinterpret_cast<V2*>(f.v1 + idx) = V2{ov[0], ov[1]};
        } else {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (okmask & (1u << k)) {
                    f.eta1[idx + k] = oe[k];
                    f.u1[idx + k] = ou[k];
                    f.v1[idx + k] = ov[k];
                }
            }
        }
    }
    // ---- phase C: Dirichlet nodes of this tile
    if (dir_start) {
        const int b = dir_start[tile], e = dir_start[tile + 1];
        if (b < e) {
            __syncthreads();  // the block's new values are visible to the block
            for (int k = b + (int)threadIdx.x; k < e; k += THREADS)
                dirichlet_node(f.eta1, f.u1, f.v1, f.D, D64, dir_list[k], bv);
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 tile phase A with paired arithmetic: a thread's two nodes of a row
// are the two lanes of every operation of derive.  Same operations, same
// results as tile_phase_a.
__device__ __forceinline__ void store_pair2(tile::Derived<float>& sm, int pr, int lc, const Src2& s)
{
    const float2 od[8] = {s.o1, s.o2, s.o3, s.o4, s.o5, s.o6, s.o7, s.o8};
#pragma unroll
    for (int d = 0; d < 8; ++d) *reinterpret_cast<float2*>(&sm.o(d, pr, lc)) = od[d];
    sm.ed(pr, lc) = make_float2(s.eta.x, s.D.x);
    sm.ed(pr, lc + 1) = make_float2(s.eta.y, s.D.y);
}

template <int FM>
__device__ __forceinline__ void tile_phase_a_f32(const Fields<float>& f, int x0, int y0, bool inside,
                                                 const tma::Stage* st, tile::Derived<float>& sm, Src2 (&own)[2],
                                                 uint32_t (&own_types)[2])
{
    using namespace tile;
    const int tx = threadIdx.x & 31, tyy = threadIdx.x >> 5;
    Raw<float> raw[2][2];
    Raw<float> hraw[2];
    uint32_t htypes;
    int hpr = 0, hpc = 0;
    const bool has_halo = threadIdx.x < HALO_PAIRS;
    if (has_halo) {
        const int h = threadIdx.x;
        if (h < 2 * IR) { hpc = h < IR ? 0 : PC - 1; hpr = h % IR; }
        else { const int u = h - 2 * IR; hpr = u < PC - 2 ? 0 : IR - 1; hpc = 1 + u % (PC - 2); }
    }
    if (st) {
#pragma unroll
        for (int r = 0; r < 2; ++r) staged_pair(*st, 1 + 2 * tyy + r, 2 + 2 * tx, raw[r], own_types[r]);
        if (has_halo) staged_pair(*st, hpr, 2 * hpc, hraw, htypes);
    } else if (inside) {
        const int off = (y0 + 2 * tyy) * f.pitch + x0 + 2 * tx;
        load_pair_in(f, off, raw[0], own_types[0]);
        load_pair_in(f, off + f.pitch, raw[1], own_types[1]);
        if (has_halo) load_pair_in(f, (y0 - 1 + hpr) * f.pitch + x0 - 2 + 2 * hpc, hraw, htypes);
    } else {
#pragma unroll
        for (int r = 0; r < 2; ++r) load_pair(f, y0 + 2 * tyy + r, x0 + 2 * tx, raw[r], own_types[r]);
        if (has_halo) load_pair(f, y0 - 1 + hpr, x0 - 2 + 2 * hpc, hraw, htypes);
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        derive2<FM>(coef2_of(f.c), raw[r][0], raw[r][1], own[r]);
        store_pair2(sm, 1 + 2 * tyy + r, 2 + 2 * tx, own[r]);
    }
    if (has_halo) {
        Src2 hs;
        derive2<FM>(coef2_of(f.c), hraw[0], hraw[1], hs);
        store_pair2(sm, hpr, 2 * hpc, hs);
    }
}

__device__ __forceinline__ Src<float> lane_of(const Src2& s, int k)
{
    Src<float> o;
#define MACLAB_LANE(m) o.m = k ? s.m.y : s.m.x;
    MACLAB_LANE(eta) MACLAB_LANE(D) MACLAB_LANE(o1) MACLAB_LANE(o2) MACLAB_LANE(o3) MACLAB_LANE(o4)
    MACLAB_LANE(o5) MACLAB_LANE(o6) MACLAB_LANE(o7) MACLAB_LANE(o8) MACLAB_LANE(ownh) MACLAB_LANE(hFx)
    MACLAB_LANE(hFy)
#undef MACLAB_LANE
    return o;
}

__device__ __forceinline__ void tile_phase_bc_f32(const Fields<float>& f, int x0, int y0, bool inside, int tile,
                                                  const int* dir_start, const DirNode* dir_list, const double* D64,
                                                  const DirValues& bv, const tile::Derived<float>& sm,
                                                  const Src2 (&own)[2], const uint32_t (&own_types)[2])
{
    // phase B stays one node per instruction: pairing it needs the
    // neighbours' (eta, D) regrouped by lane, which costs more moves and
    // loads than the paired arithmetic saves
    const Src<float> o[2][2] = {{lane_of(own[0], 0), lane_of(own[0], 1)}, {lane_of(own[1], 0), lane_of(own[1], 1)}};
    tile_phase_bc<float>(f, x0, y0, inside, tile, dir_start, dir_list, D64, bv, sm, o, own_types);
}

// Update of one tile whose top-left updated node is (x0, y0); `tile` indexes
// the per-tile Dirichlet ranges and, when gstart is given, the per-tile
// ranges of glist: the tile's nodes with a bounce-back link, updated here by
// the per-link form (they read only the old state and no other node of the
// step reads their new values before the next step, so no barrier is needed).
template <typename T, int FM>
__device__ __forceinline__ void tile_update(const Fields<T>& f, int x0, int y0, int tile, const int* dir_start,
                                            const DirNode* dir_list, const double* D64, const DirValues& bv,
                                            tile::Derived<T>& sm, const int* gstart = nullptr,
                                            const int* glist = nullptr)
{
    uint32_t own_types[2];
    const bool inside = tile_inside(f, x0, y0);
    if constexpr (std::is_same<T, float>::value) {
        Src2 own[2];
        tile_phase_a_f32<FM>(f, x0, y0, inside, nullptr, sm, own, own_types);
        __syncthreads();
        tile_phase_bc_f32(f, x0, y0, inside, tile, dir_start, dir_list, D64, bv, sm, own, own_types);
    } else {
        Src<T> own[2][2];
        tile_phase_a<T, FM>(f, x0, y0, inside, sm, own, own_types);
        __syncthreads();
        tile_phase_bc<T>(f, x0, y0, inside, tile, dir_start, dir_list, D64, bv, sm, own, own_types);
    }
    if (gstart) {
        const int e = gstart[tile + 1];
        for (int k = gstart[tile] + (int)threadIdx.x; k < e; k += tile::THREADS) {
            const int node = glist[k];
            general_node<T>(f, node % f.nx, node / f.nx);
        }
    }
}

template <typename T, int FM>
__global__ void __launch_bounds__(tile::THREADS, tile::MinBlocks<T>::value)
step_tile_kernel(const __grid_constant__ Fields<T> f, int tiles_x, int tiles_y, const __grid_constant__ TileDirichlet td)
{
    // block (bx, by, bz) updates tile column bx of tile row bz * gridDim.y + by
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile::Derived<T>& sm = *reinterpret_cast<tile::Derived<T>*>(smem_raw);
    const int ty = blockIdx.z * gridDim.y + blockIdx.y;
    if (ty >= tiles_y) return;  // whole block
    tile_update<T, FM>(f, blockIdx.x * tile::TX, ty * tile::TY, ty * tiles_x + blockIdx.x, td.start, td.list, td.D64,
                       td.bv, sm, td.gstart, td.glist);
}

// Single step over a list of tiles (the tiles a two-step launch leaves out).
template <typename T, int FM>
__global__ void __launch_bounds__(tile::THREADS, tile::MinBlocks<T>::value)
step_tile_list_kernel(const __grid_constant__ Fields<T> f, int tiles_x, const __grid_constant__ TileDirichlet td,
                      const int* __restrict__ list)
{
    extern __shared__ __align__(16) unsigned char smem_list[];
    tile::Derived<T>& sm = *reinterpret_cast<tile::Derived<T>*>(smem_list);
    const int t = list[blockIdx.x];
    const int x0 = (t % tiles_x) * tile::TX, y0 = (t / tiles_x) * tile::TY;
    tile_update<T, FM>(f, x0, y0, t, td.start, td.list, td.D64, td.bv, sm, td.gstart, td.glist);
}

// ---------------------------------------------------------------------------
// Two steps per launch (temporal blocking, FP32) for "clean" tiles: the
// 68 x 20 window of the tile (two nodes of halo on every side) lies inside
// the grid and holds only fluid and no-slip nodes without bounce-back links,
// so no edge rule, bounce-back link or Dirichlet node enters either step.
//   A1  derive the window at step n           (rows 0..19 of the window)
//   B1  update rows 1..18 to step n + 1, kept in registers; the tile's
//       outer ring of nodes is also written to the step-n+1 buffer for the
//       tiles that take two single steps
//   A2  derive those rows at step n + 1
//   B2  update the 64 x 16 tile to step n + 2 and store it
// Window column c is global x0 - 2 + c, window row r global y0 - 2 + r.
// Every node value equals that of two single steps bitwise (same
// derive2 / node_update arithmetic).
namespace tile2 {
constexpr int R2 = tile::TY + 4;            // 20 window rows
constexpr int PAIRS = R2 * tile::PC;        // 680 pairs of the window
constexpr int MID = (R2 - 2) * tile::PC;    // 612 pairs of rows 1..18
constexpr int HOLD = (MID + tile::THREADS - 1) / tile::THREADS;  // 3
struct Smem {
    tile::Derived<float, R2> d;
    float2 own[3][R2][tile::PC];            // ownh, hFx, hFy of pair (r, j): columns 2j, 2j + 1
    uint16_t type[R2][tile::PC];
};
}  // namespace tile2

__device__ __forceinline__ void store_window_pair(tile2::Smem& sm, int r, int j, const Src2& s, uint32_t types)
{
    const float2 od[8] = {s.o1, s.o2, s.o3, s.o4, s.o5, s.o6, s.o7, s.o8};
#pragma unroll
    for (int d = 0; d < 8; ++d) *reinterpret_cast<float2*>(&sm.d.o(d, r, 2 * j)) = od[d];
    sm.d.ed(r, 2 * j) = make_float2(s.eta.x, s.D.x);
    sm.d.ed(r, 2 * j + 1) = make_float2(s.eta.y, s.D.y);
    sm.own[0][r][j] = s.ownh;
    sm.own[1][r][j] = s.hFx;
    sm.own[2][r][j] = s.hFy;
    sm.type[r][j] = (uint16_t)types;
}

__device__ __forceinline__ void window_node(const tile2::Smem& sm, const Coef<float>& K, int r, int c, float& oe,
                                            float& ou, float& ov)
{
    const int j = c >> 1, k = c & 1;
    const float2 ed = sm.d.ed(r, c);
    const float2 oh = sm.own[0][r][j], fx = sm.own[1][r][j], fy = sm.own[2][r][j];
    const uint8_t ty = (uint8_t)(sm.type[r][j] >> (8 * k));
    node_update<float>(sm.d, r, c, K, ed.x, ed.y, k ? oh.y : oh.x, k ? fx.y : fx.x, k ? fy.y : fy.x,
                       (ty & KIND_MASK) == K_NOSLIP, oe, ou, ov);
}

// f: eta, u, v at step n; eta1, u1, v1 the step-n+1 buffer (outer ring only);
// out_* the step-n+2 buffer.  Blocks walk the list of clean tiles.
template <int FM>
__global__ void __launch_bounds__(tile::THREADS, 3)
step_tile2_kernel(const __grid_constant__ Fields<float> f, float* __restrict__ out_eta, float* __restrict__ out_u,
                  float* __restrict__ out_v, int tiles_x, const int* __restrict__ list)
{
    using namespace tile;
    using namespace tile2;
    extern __shared__ __align__(16) unsigned char smem_t2[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_t2);
    const int t = list[blockIdx.x];
    const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
    const Coef<float>& K = f.c;
    // ---- A1: the window at step n (inside the grid: plain vector loads)
    for (int p = threadIdx.x; p < PAIRS; p += THREADS) {
        const int r = p / PC, j = p % PC;
        const size_t base = (size_t)(y0 - 2 + r) * f.pitch + x0 - 2 + 2 * j;
        const float2 e2 = *reinterpret_cast<const float2*>(f.eta + base);
        const float2 u2 = *reinterpret_cast<const float2*>(f.u + base);
        const float2 v2 = *reinterpret_cast<const float2*>(f.v + base);
        const float2 d2 = *reinterpret_cast<const float2*>(f.D + base);
        const uint32_t types = *reinterpret_cast<const uint16_t*>(f.type + base);
        Src2 s;
        derive2<FM>(coef2_of(K), Raw<float>{e2.x, u2.x, v2.x, d2.x, 0}, Raw<float>{e2.y, u2.y, v2.y, d2.y, 0}, s);
        store_window_pair(sm, r, j, s, types);
    }
    __syncthreads();
    // ---- B1: rows 1..18 at step n + 1 (window columns 0 and 67 have no
    // update; they are computed from in-window neighbours and never read)
    float2 he[HOLD], hu[HOLD], hv[HOLD], hd[HOLD];
    uint32_t ht[HOLD];
#pragma unroll
    for (int k = 0; k < HOLD; ++k) {
        const int p = threadIdx.x + k * THREADS;
        if (p >= MID) break;
        const int r = 1 + p / PC, j = p % PC;
        float oe[2], ou[2], ov[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int c = min(max(2 * j + l, 1), IW - 2);
            window_node(sm, K, r, c, oe[l], ou[l], ov[l]);
            // outer ring of the tile -> the step-n+1 buffer
            const int cc = 2 * j + l;
            if (r >= 2 && r <= R2 - 3 && cc >= 2 && cc <= IW - 3 &&
                (r == 2 || r == R2 - 3 || cc == 2 || cc == IW - 3)) {
                const size_t idx = (size_t)(y0 - 2 + r) * f.pitch + x0 - 2 + cc;
                f.eta1[idx] = oe[l];
                f.u1[idx] = ou[l];
                f.v1[idx] = ov[l];
            }
        }
        he[k] = make_float2(oe[0], oe[1]);
        hu[k] = make_float2(ou[0], ou[1]);
        hv[k] = make_float2(ov[0], ov[1]);
        hd[k] = make_float2(sm.d.ed(r, 2 * j).y, sm.d.ed(r, 2 * j + 1).y);
        ht[k] = sm.type[r][j];
    }
    __syncthreads();
    // ---- A2: derive rows 1..18 at step n + 1
#pragma unroll
    for (int k = 0; k < HOLD; ++k) {
        const int p = threadIdx.x + k * THREADS;
        if (p >= MID) break;
        const int r = 1 + p / PC, j = p % PC;
        Src2 s;
        derive2<FM>(coef2_of(K), Raw<float>{he[k].x, hu[k].x, hv[k].x, hd[k].x, 0},
                    Raw<float>{he[k].y, hu[k].y, hv[k].y, hd[k].y, 0}, s);
        store_window_pair(sm, r, j, s, ht[k]);
    }
    __syncthreads();
    // ---- B2: the tile (window rows 2..17, columns 2..65) at step n + 2
    const int tx = threadIdx.x & 31, tyy = threadIdx.x >> 5;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int r = 2 + 2 * tyy + rr;
        float oe[2], ou[2], ov[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) window_node(sm, K, r, 2 + 2 * tx + l, oe[l], ou[l], ov[l]);
        const size_t idx = (size_t)(y0 - 2 + r) * f.pitch + x0 + 2 * tx;
        *reinterpret_cast<float2*>(out_eta + idx) = make_float2(oe[0], oe[1]);
        *reinterpret_cast<float2*>(out_u + idx) = make_float2(ou[0], ou[1]);
        *reinterpret_cast<float2*>(out_v + idx) = make_float2(ov[0], ov[1]);
    }
}

// ---------------------------------------------------------------------------
// TMA-staged tile kernel (FP32).  Blocks are persistent (three per SM) and
// walk the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  The raw rows of an
// interior tile (every row and column its phase A reads lies inside the
// grid, so no edge rule applies) arrive in shared memory by five 2D tensor
// copies that one thread issues while the block still works on the previous
// tile's gather; an mbarrier counts the bytes.  Edge tiles load through the
// edge rules as in step_tile_kernel.  Every mbarrier wait is bounded: on
// timeout the block sets *err, waits (bounded again) for its copy and leaves.
struct TmaMaps {
    CUtensorMap eta, u, v, D, type;   // 2D maps of the state being read, D and the types
};
constexpr uint32_t TMA_WAIT_LIMIT = 1u << 22;   // try_wait rounds before giving up

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase of parity `phase` has completed; false after `limit` rounds
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, uint32_t limit)
{
    for (uint32_t k = 0; k < limit; ++k) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// Stage the rows of the tile at (x0, y0).  x0 is a multiple of 64, so both
// inner coordinates (x0 - 4 floats, x0 - 16 bytes) start on 16 bytes.
__device__ __forceinline__ void tma_stage(const TmaMaps& m, tma::Stage& st, uint32_t bar, int x0, int y0)
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // earlier reads of the buffer come first
    mbar_expect_tx(bar, tma::BYTES);
    tma_load_2d((uint32_t)__cvta_generic_to_shared(&st.f[0][0]), &m.eta, x0 - 4, y0 - 1, bar);
    tma_load_2d((uint32_t)__cvta_generic_to_shared(&st.f[1][0]), &m.u, x0 - 4, y0 - 1, bar);
    tma_load_2d((uint32_t)__cvta_generic_to_shared(&st.f[2][0]), &m.v, x0 - 4, y0 - 1, bar);
    tma_load_2d((uint32_t)__cvta_generic_to_shared(&st.f[3][0]), &m.D, x0 - 4, y0 - 1, bar);
    tma_load_2d((uint32_t)__cvta_generic_to_shared(&st.type[0]), &m.type, x0 - 16, y0 - 1, bar);
}
template <int FM>
__global__ void __launch_bounds__(tile::THREADS, 3)
step_tile_tma_kernel(const __grid_constant__ Fields<float> f, const __grid_constant__ TmaMaps maps, int tiles_x,
                     int ntiles, const __grid_constant__ TileDirichlet td, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_tma[];
    // the base rounded up to 128 bytes (tma::SMEM holds the slack)
    unsigned char* base = smem_tma + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_tma) & 127u)) & 127u);
    tile::Derived<float>& sm = *reinterpret_cast<tile::Derived<float>*>(base);
    tma::Stage& st = *reinterpret_cast<tma::Stage*>(base + tma::STAGE_OFF);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int abort_flag;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    int t = blockIdx.x;
    if (threadIdx.x == 0 && t < ntiles) {
        const int x0 = (t % tiles_x) * tile::TX, y0 = (t / tiles_x) * tile::TY;
        if (tile_interior(f.nx, f.ny, x0, y0)) tma_stage(maps, st, bar, x0, y0);
    }
    for (; t < ntiles; t += gridDim.x) {
        const int x0 = (t % tiles_x) * tile::TX, y0 = (t / tiles_x) * tile::TY;
        const bool staged = tile_interior(f.nx, f.ny, x0, y0);
        if (staged) {
            if (!mbar_wait(bar, phase, TMA_WAIT_LIMIT)) atomicOr(&abort_flag, 1);
            __syncthreads();
            if (abort_flag) {
                if (threadIdx.x == 0) atomicOr(err, 1);
                mbar_wait(bar, phase, TMA_WAIT_LIMIT);  // the copy lands before the block leaves
                return;
            }
            phase ^= 1u;
        }
        Src2 own[2];
        uint32_t own_types[2];
        tile_phase_a_f32<FM>(f, x0, y0, false, staged ? &st : nullptr, sm, own, own_types);
        __syncthreads();  // derived values visible; the staging buffer is free again
        if (threadIdx.x == 0) {
            const int tn = t + gridDim.x;
            if (tn < ntiles) {
                const int xn = (tn % tiles_x) * tile::TX, yn = (tn / tiles_x) * tile::TY;
                if (tile_interior(f.nx, f.ny, xn, yn)) tma_stage(maps, st, bar, xn, yn);
            }
        }
        tile_phase_bc_f32(f, x0, y0, staged && f.idx32, t, td.start, td.list, td.D64, td.bv, sm, own, own_types);
        __syncthreads();  // phase B reads of `sm` end before the next phase A writes it
    }
}

// ---------------------------------------------------------------------------
// Batched step: one launch advances every active instance of a batch.  The
// tiles of all instances form one list; block b updates tile tile_local[b]
// of instance tile_inst[b] with that instance's fields and coefficients.
// Instances whose flag in `active` is 0 are skipped (their state stays).
template <typename T>
struct BatchInst {
    Fields<T> f[2];     // fields for the two buffer parities
    int tiles_x;        // tiles per row of the instance
    int tile0;          // index of the instance's first tile in the batch list
    int ntiles;         // tiles of the instance
    int pad;
    const double* D64;  // still-water depth in double (Dirichlet depths)
    DirValues bv;       // steady Dirichlet values
};

template <typename T>
__global__ void __launch_bounds__(tile::THREADS, tile::BatchMinBlocks<T>::value)
step_batch_kernel(const BatchInst<T>* __restrict__ insts, const int* __restrict__ tile_inst,
                  const uint8_t* __restrict__ active, int parity, const int* __restrict__ dir_start,
                  const DirNode* __restrict__ dirs, const int* __restrict__ gstart, const int* __restrict__ glist)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile::Derived<T>& sm = *reinterpret_cast<tile::Derived<T>*>(smem_raw);
    const int i = tile_inst[blockIdx.x];
    if (!active[i]) return;  // whole block
    const BatchInst<T>& in = insts[i];
    const Fields<T> f = in.f[parity];
    const int t = blockIdx.x - in.tile0;
    const int x0 = (t % in.tiles_x) * tile::TX, y0 = (t / in.tiles_x) * tile::TY;
    // all force terms: absent ones have zero coefficients and contribute
    // exact zeros, so every instance gets the same values as its own kernel
    tile_update<T, F_WIND | F_FRICTION | F_CORIOLIS>(f, x0, y0, blockIdx.x, dir_start, dirs, in.D64, in.bv, sm,
                                                     gstart, glist);
}

// Nodes with a bounce-back link across a batch: (instance, node) pairs.
template <typename T>
__global__ void __launch_bounds__(128) batch_general_kernel(const BatchInst<T>* __restrict__ insts,
                                                            const int2* __restrict__ list, int count,
                                                            const uint8_t* __restrict__ active, int parity)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int2 e = list[t];
    if (!active[e.x]) return;
    const Fields<T>& f = insts[e.x].f[parity];
    general_node(f, e.y % f.nx, e.y / f.nx);
}

// Dirichlet nodes across a batch (when they cannot be fused into the tiles):
// (instance, index into the batch list) pairs.
template <typename T>
__global__ void batch_dirichlet_kernel(const BatchInst<T>* __restrict__ insts, const int* __restrict__ owner,
                                       const DirNode* __restrict__ dirs, int count,
                                       const uint8_t* __restrict__ active, int parity)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int i = owner[t];
    if (!active[i]) return;
    const BatchInst<T>& in = insts[i];
    const Fields<T>& f = in.f[parity];
    dirichlet_node(f.eta1, f.u1, f.v1, f.D, in.D64, dirs[t], in.bv);
}

// ---------------------------------------------------------------------------
// Persistent batched steps.  One cooperative launch of G blocks (all
// resident at once, which the cooperative launch guarantees or refuses)
// runs `nsteps` steps of the batch: in each step block b updates the tiles
// b, b + G, ... of the packed list and a grid-stride share of the
// bounce-back-link nodes (both read only the old state), then every block
// meets at a grid barrier; Dirichlet nodes that could not be fused into
// their tiles follow, with a second barrier.  The work of a step is that of
// step_batch_kernel, batch_general_kernel and batch_dirichlet_kernel, so the
// results are the same bitwise.
//
// Grid barrier: a counter and a generation word in device memory.  Thread 0
// of each block publishes its block's writes (__threadfence), counts itself
// in; the last to arrive resets the counter and advances the generation, the
// others poll it.  The launch's first generation comes from the host, which
// counts the barriers it has launched.  Every poll is bounded: after
// BARRIER_POLLS rounds the block sets *err and reports failure, and the
// kernel's blocks leave instead of stepping on.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};
constexpr unsigned int BARRIER_POLLS = 1u << 22;

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// true when every block has arrived; `gen` is this block's count of the
// barriers passed so far (it advances by one)
__device__ __forceinline__ bool grid_barrier(GridBarrier* gb, unsigned int nblocks, unsigned int& gen, int* err,
                                             unsigned int polls)
{
    __shared__ int gb_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned int g = gen;
        if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicExch(&gb->gen, g + 1);
        } else {
            unsigned int k = 0;
            while (ld_acquire_gpu(&gb->gen) == g) {
                if (++k >= polls) {
                    atomicOr(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gb_ok = ok;
    }
    __syncthreads();
    gen += 1;
    return gb_ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(tile::THREADS, tile::BatchMinBlocks<T>::value)
step_batch_persistent_kernel(const BatchInst<T>* __restrict__ insts, const int* __restrict__ tile_inst, int ntiles,
                             const uint8_t* __restrict__ active, int parity, int nsteps,
                             const int* __restrict__ dir_start, const DirNode* __restrict__ dirs,
                             const int2* __restrict__ general, int n_general, const int* __restrict__ dir_owner,
                             int n_dir_sep, GridBarrier* gb, unsigned int gen, int* err, unsigned int nbar,
                             unsigned int polls)
{
    extern __shared__ __align__(16) unsigned char smem_persist[];
    tile::Derived<T>& sm = *reinterpret_cast<tile::Derived<T>*>(smem_persist);
    const unsigned int G = gridDim.x;
    const int gthreads = (int)(G * blockDim.x), gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    for (int s = 0; s < nsteps; ++s, parity ^= 1) {
        for (int t = blockIdx.x; t < ntiles; t += G) {
            const int i = tile_inst[t];
            if (!active[i]) continue;  // whole block
            const BatchInst<T>& in = insts[i];
            const Fields<T> f = in.f[parity];
            const int tl = t - in.tile0;
            const int x0 = (tl % in.tiles_x) * tile::TX, y0 = (tl / in.tiles_x) * tile::TY;
            tile_update<T, F_WIND | F_FRICTION | F_CORIOLIS>(f, x0, y0, t, dir_start, dirs, in.D64, in.bv, sm);
            __syncthreads();  // the gather's reads end before the next tile's derivation writes
        }
        for (int k = gtid; k < n_general; k += gthreads) {
            const int2 e = general[k];
            if (!active[e.x]) continue;
            const Fields<T>& f = insts[e.x].f[parity];
            general_node(f, e.y % f.nx, e.y / f.nx);
        }
        if (!grid_barrier(gb, nbar, gen, err, polls)) return;
        if (n_dir_sep > 0) {
            for (int k = gtid; k < n_dir_sep; k += gthreads) {
                const int i = dir_owner[k];
                if (!active[i]) continue;
                const BatchInst<T>& in = insts[i];
                const Fields<T>& f = in.f[parity];
                dirichlet_node(f.eta1, f.u1, f.v1, f.D, in.D64, dirs[k], in.bv);
            }
            if (!grid_barrier(gb, nbar, gen, err, polls)) return;
        }
    }
}

// ---------------------------------------------------------------------------
// Residual / mass / stability reduction in double precision.
constexpr int RED_THREADS = 256;
constexpr int RED_NVAL = 5;  // sum dq^2, sum q^2, sum eta, max |u|^2, non-finite count

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_max(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
residual_partial_kernel(const T* __restrict__ e0, const T* __restrict__ u0, const T* __restrict__ v0,
                        const T* __restrict__ e1, const T* __restrict__ u1, const T* __restrict__ v1,
                        const T* __restrict__ D, const uint8_t* __restrict__ type, int nx, int ny,
                        int pitch, double* __restrict__ partial)
{
    double s[RED_NVAL] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const size_t total = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
         k += (size_t)gridDim.x * blockDim.x) {
        const size_t j = k / nx, i = k - j * nx;
        const size_t x = j * pitch + i;
        if ((type[x] & KIND_MASK) == K_SOLID) continue;
        const double d = (double)D[x];
        const double a0 = (double)e0[x], a1 = (double)e1[x];
        const double h0 = d + a0, h1 = d + a1;
        const double qx0 = h0 * (double)u0[x], qy0 = h0 * (double)v0[x];
        const double qx1 = h1 * (double)u1[x], qy1 = h1 * (double)v1[x];
        const double dh = a1 - a0, dqx = qx1 - qx0, dqy = qy1 - qy0;
        s[0] += dh * dh + dqx * dqx + dqy * dqy;
        s[1] += h1 * h1 + qx1 * qx1 + qy1 * qy1;
        s[2] += a1;
        const double uu = (double)u1[x] * (double)u1[x] + (double)v1[x] * (double)v1[x];
        s[3] = fmax(s[3], uu);
        if (!isfinite(a1) || !isfinite(uu)) s[4] += 1.0;
    }
    __shared__ double sh[RED_NVAL][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < RED_NVAL; ++q) {
        const double r = (q == 3) ? warp_max(s[q]) : warp_sum(s[q]);
        if (lane == 0) sh[q][w] = r;
    }
    __syncthreads();
    if (threadIdx.x < RED_NVAL) {
        const int q = threadIdx.x;
        double r = sh[q][0];
        for (int k = 1; k < RED_THREADS / 32; ++k) r = (q == 3) ? fmax(r, sh[q][k]) : r + sh[q][k];
        partial[(size_t)blockIdx.x * RED_NVAL + q] = r;
    }
}

__global__ void residual_final_kernel(const double* __restrict__ partial, int nblocks,
                                      double* __restrict__ out)
{
    // one warp per value, fixed order -> deterministic
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= RED_NVAL) return;
    double r = (q == 3) ? 0.0 : 0.0;
    for (int b = lane; b < nblocks; b += 32) {
        const double x = partial[(size_t)b * RED_NVAL + q];
        r = (q == 3) ? fmax(r, x) : r + x;
    }
    r = (q == 3) ? warp_max(r) : warp_sum(r);
    if (lane == 0) out[q] = r;
}

// Per-instance residual of a batch: block b sums the nodes of tile b of its
// instance (old state = parity buffers, new = the other ones) into
// partial[b][RED_NVAL]; then one warp per instance adds its tiles in order.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
batch_residual_tile_kernel(const BatchInst<T>* __restrict__ insts, const int* __restrict__ tile_inst,
                           int parity, double* __restrict__ partial, const T* se, const T* su, const T* sv,
                           const T* ce, const T* cu, const T* cv)
{
    const int i = tile_inst[blockIdx.x];
    const BatchInst<T>& in = insts[i];
    const Fields<T>& f = in.f[parity];  // eta = previous state, eta1 = current state
    // with a marked state (se != nullptr): the previous state is the mark,
    // laid out like the current buffer (ce, cu, cv: its bases)
    const T* pe = se ? se + (f.eta1 - ce) : f.eta;
    const T* pu = se ? su + (f.u1 - cu) : f.u;
    const T* pv = se ? sv + (f.v1 - cv) : f.v;
    const int t = blockIdx.x - in.tile0;
    const int x0 = (t % in.tiles_x) * tile::TX, y0 = (t / in.tiles_x) * tile::TY;
    double s[RED_NVAL] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < tile::TX * tile::TY; k += RED_THREADS) {
        const int x = x0 + (k % tile::TX), y = y0 + k / tile::TX;
        if (x >= f.nx || y >= f.ny) continue;
        const size_t p = (size_t)y * f.pitch + x;
        if ((f.type[p] & KIND_MASK) == K_SOLID) continue;
        const double d = (double)f.D[p];
        const double a0 = (double)pe[p], a1 = (double)f.eta1[p];
        const double h0 = d + a0, h1 = d + a1;
        const double qx0 = h0 * (double)pu[p], qy0 = h0 * (double)pv[p];
        const double qx1 = h1 * (double)f.u1[p], qy1 = h1 * (double)f.v1[p];
        const double dh = a1 - a0, dqx = qx1 - qx0, dqy = qy1 - qy0;
        s[0] += dh * dh + dqx * dqx + dqy * dqy;
        s[1] += h1 * h1 + qx1 * qx1 + qy1 * qy1;
        s[2] += a1;
        const double uu = (double)f.u1[p] * (double)f.u1[p] + (double)f.v1[p] * (double)f.v1[p];
        s[3] = fmax(s[3], uu);
        if (!isfinite(a1) || !isfinite(uu)) s[4] += 1.0;
    }
    __shared__ double sh[RED_NVAL][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < RED_NVAL; ++q) {
        const double r = (q == 3) ? warp_max(s[q]) : warp_sum(s[q]);
        if (lane == 0) sh[q][w] = r;
    }
    __syncthreads();
    if (threadIdx.x < RED_NVAL) {
        const int q = threadIdx.x;
        double r = sh[q][0];
        for (int k = 1; k < RED_THREADS / 32; ++k) r = (q == 3) ? fmax(r, sh[q][k]) : r + sh[q][k];
        partial[(size_t)blockIdx.x * RED_NVAL + q] = r;
    }
}

template <typename T>
__global__ void batch_residual_final_kernel(const BatchInst<T>* __restrict__ insts, int count,
                                            const double* __restrict__ partial, double* __restrict__ out)
{
    const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= count) return;
    const int t0 = insts[i].tile0, nt = insts[i].ntiles;
#pragma unroll 1
    for (int q = 0; q < RED_NVAL; ++q) {
        double r = 0.0;
        for (int b = lane; b < nt; b += 32) {
            const double x = partial[(size_t)(t0 + b) * RED_NVAL + q];
            r = (q == 3) ? fmax(r, x) : r + x;
        }
        r = (q == 3) ? warp_max(r) : warp_sum(r);
        if (lane == 0) out[(size_t)i * RED_NVAL + q] = r;
    }
}

// ---------------------------------------------------------------------------
// State conversion between host-facing double (h, u, v) [ny][nx] and the
// device storage (eta, u, v) [ny][pitch].
template <typename T>
__global__ void state_in_kernel(const double* __restrict__ h, const double* __restrict__ u,
                                const double* __restrict__ v, const double* __restrict__ D64,
                                const uint8_t* __restrict__ type, T* e0, T* u0, T* v0, T* e1,
                                T* u1, T* v1, int nx, int ny, int pitch)
{
    const size_t total = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
         k += (size_t)gridDim.x * blockDim.x) {
        const size_t j = k / nx, i = k - j * nx, x = j * pitch + i;
        const T a = (T)(h[k] - D64[x]), b = (T)u[k], c = (T)v[k];
        e0[x] = a; u0[x] = b; v0[x] = c;
        if ((type[x] & KIND_MASK) == K_SOLID) { e1[x] = a; u1[x] = b; v1[x] = c; }
    }
}

template <typename T>
__global__ void state_out_kernel(const T* __restrict__ e, const T* __restrict__ u,
                                 const T* __restrict__ v, const double* __restrict__ D64,
                                 double* h, double* uo, double* vo, int nx, int ny, int pitch)
{
    const size_t total = (size_t)nx * ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
         k += (size_t)gridDim.x * blockDim.x) {
        const size_t j = k / nx, i = k - j * nx, x = j * pitch + i;
        h[k] = D64[x] + (double)e[x];
        uo[k] = (double)u[x];
        vo[k] = (double)v[x];
    }
}

}  // namespace maclab
