// maclab_elab.cuh -- device code of the eLABSWE distribution form with a
// general relaxation time (Zhou, arXiv:1902.02999, Eq. lb.1) for sm_103a;
// included after maclab_kernels.cuh, whose tile geometry, edge rules and
// coefficients it shares.
#pragma once
#include "maclab_kernels.cuh"

namespace maclab {

// ---------------------------------------------------------------------------
// eLABSWE with a general relaxation time tau (Eq. lb.1): nine distributions
// per node, stored as g_a = f_a - f^eq_a(D, 0) (perturbations about the rest
// equilibrium, so that a lake at rest is g = 0 exactly).  In these variables
// one step of Eq. lb.1, pulled at node x from y = x - c_a, reads
//   g_a(x, t + dt) = g*_a(y) + lambda_a [ -G6 (eta_x + eta_y)(D_y - D_x)
//                                          + KF c_a . (F_x + F_y) ]
//   g*_a(y)        = g_a(y) + (o_a(y) - g_a(y)) / tau,
//   o_a            = f^eq_a(h, u) - f^eq_a(D, 0)      (Eq. feq-full),
// the rest-equilibrium difference f^eq_a(D_y, 0) - f^eq_a(D_x, 0) having
// cancelled the D-only part of the bed term.  A source that is solid or
// behind a bounce-back edge gives g*_abar(x); a specular source is the
// mirror node, supplying g*_{mirror(a)} there with its force mirrored.
// h = D + sum_a g_a and h u = e sum_a c_a g_a (Eqs. fea-0-h, fea-0-v).
// A block owns a 64 x 16 tile; phase A collides the tile and its one-node
// halo into shared memory, phase B streams.  Tiles inside the grid skip the
// edge rules; FP32 takes the reciprocal of h from the hardware approximation
// (about 1 ulp), as the macroscopic kernels do.
namespace elab {
template <typename T>
struct Smem {
    T gs[9][tile::IR][tile::IW];                   // post-collision g*, direction-mapped for mirrors
    typename Vec2<T>::type ed[tile::IR][tile::IW]; // (eta, D)
    typename Vec2<T>::type F[tile::IR][tile::IW];  // KF F (source half already in gs)
    uint8_t use[tile::IR][tile::IW];               // usable source
};
template <typename T> struct MinBlocks { static constexpr int value = 3; };
template <> struct MinBlocks<double> { static constexpr int value = 1; };
}  // namespace elab

// Lattice vectors as compile-time values: in unrolled loops over the
// directions they fold into the arithmetic.
__host__ __device__ constexpr int lat_cx(int a) { return (a == 1 || a == 2 || a == 8) ? 1 : (a >= 4 && a <= 6) ? -1 : 0; }
__host__ __device__ constexpr int lat_cy(int a) { return (a >= 2 && a <= 4) ? 1 : (a >= 6) ? -1 : 0; }
__host__ __device__ constexpr int lat_dir(int cx, int cy)
{
    return cx == 0 ? (cy == 0 ? 0 : cy > 0 ? 3 : 7) : cx > 0 ? (cy == 0 ? 1 : cy > 0 ? 2 : 8) : (cy == 0 ? 5 : cy > 0 ? 4 : 6);
}
// direction with lattice vector (sx c_x, sy c_y), sx = -1 for mirror bit 1,
// sy = -1 for mirror bit 2 (b known at compile time, fl at run time)
__device__ __forceinline__ int mirror_of(int b, uint8_t fl)
{
    const int mx = lat_dir(-lat_cx(b), lat_cy(b)), my = lat_dir(lat_cx(b), -lat_cy(b));
    const int mxy = lat_dir(-lat_cx(b), -lat_cy(b));
    return fl == 1 ? mx : fl == 2 ? my : fl == 3 ? mxy : b;
}

// o_a = f^eq_a(h, u, v) - f^eq_a(D, 0), a = 0..8, and the force at a node.
// o_a = lambda_a (G6 eta (2 D + eta) - K6 h |u|^2 + h k3 (c_a.u) + h k2 (c_a.u)^2):
// opposite directions differ only in the sign of the k3 term.
template <typename T, int FM>
__device__ __forceinline__ void elab_equilibrium(const Coef<T>& c, T eta, T D, T u, T v, T (&o)[9], T& Fx, T& Fy)
{
    const T h = D + eta;
    const T uu = u * u + v * v;
    const T ge = c.G6 * eta * (T(2) * D + eta);
    const T ku = c.K6 * h * uu;
    const T gk = ge - ku;
    const T hk3 = h * c.k3, hk2 = h * c.k2;
    o[0] = eta - T(5) * ge - T(4) * ku;
    const T cu[4] = {u, u + v, v, v - u};  // c_a . u for a = 1 .. 4; a + 4 is the opposite
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T lam = (k & 1) ? T(0.25) : T(1);
        const T A = gk + hk2 * cu[k] * cu[k];
        const T B = hk3 * cu[k];
        o[k + 1] = lam * (A + B);
        o[k + 5] = lam * (A - B);
    }
    Fx = (FM & F_WIND) ? c.wfx : T(0);
    Fy = (FM & F_WIND) ? c.wfy : T(0);
    if (FM & F_CORIOLIS) {
        Fx += c.Om * h * v;
        Fy -= c.Om * h * u;
    }
    if (FM & F_FRICTION) {
        const T cbs = c.Cb * sqrt(uu);
        Fx -= cbs * u;
        Fy -= cbs * v;
    }
}

// c_a . (fx, fy) for a = 1 .. 8 (a known at compile time)
template <typename T>
__device__ __forceinline__ T lat_dot(int a, T fx, T fy)
{
    const int cx = lat_cx(a), cy = lat_cy(a);
    if (cx != 0 && cy != 0) return (cx > 0 ? fx : -fx) + (cy > 0 ? fy : -fy);
    if (cx != 0) return cx > 0 ? fx : -fx;
    return cy > 0 ? fy : -fy;
}

// Zeroth and first moments of the nine distributions.
template <typename T>
__device__ __forceinline__ void elab_moments(const T (&g)[9], T& eta, T& mx, T& my)
{
    eta = (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) + g[8];
    mx = (g[1] + g[2] + g[8]) - (g[4] + g[5] + g[6]);
    my = (g[2] + g[3] + g[4]) - (g[6] + g[7] + g[8]);
}

// gin / gout: 9 planes of [ny][pitch]; f.eta1 / u1 / v1 receive the new
// macroscopic state; omega = 1 / tau.  Block (bx, by, bz) owns tile column
// bx of tile row bz * gridDim.y + by.  The centred force term of a link,
// lambda_a KF c_a . (F_x + F_y), is split in two halves: the source half
// joins the stored post-collision value g*_a(y) (for a mirror ghost
// c_mirror(a) . F_mirrored = c_a . F, so it is formed in the node's own
// frame), the receiver half is added at x from the node's own force.  A
// bounced link takes g*_abar(x), whose source half is lambda_a KF c_abar . F_x;
// adding the receiver half lambda_a KF c_a . F_x cancels it, as the rule
// wants.
template <typename T, int FM>
__global__ void __launch_bounds__(tile::THREADS, elab::MinBlocks<T>::value)
step_elab_kernel(const __grid_constant__ Fields<T> f, const T* __restrict__ gin, T* __restrict__ gout, size_t plane,
                 T omega, int tiles_y)
{
    using namespace tile;
    using V2 = typename Vec2<T>::type;
    using O = Op<T>;
    extern __shared__ __align__(16) unsigned char smem_elab[];
    elab::Smem<T>& sm = *reinterpret_cast<elab::Smem<T>*>(smem_elab);
    const Coef<T>& K = f.c;
    const int tyi = blockIdx.z * gridDim.y + blockIdx.y;
    if (tyi >= tiles_y) return;  // whole block
    const int x0 = blockIdx.x * TX, y0 = tyi * TY;
    const bool inside = tile_inside(f, x0, y0);
    // ---- phase A: collide the tile and its halo (window rows y0-1 .. y0+16,
    // columns x0-2 .. x0+65), two window nodes per thread and round: the
    // loads of both (type, D and the nine planes) are issued before either
    // is used, so that they are in flight together
    constexpr int NA = IR * IW;
#ifndef MACLAB_ELAB_PA
#define MACLAB_ELAB_PA 3
#endif
    constexpr int PA = MACLAB_ELAB_PA;
    int all_use = 1;  // every window node this thread visits is usable
    for (int p0 = threadIdx.x; p0 < NA; p0 += PA * THREADS) {
        T g[PA][9], Dn[PA];
        uint8_t fl[PA] = {}, ty[PA] = {};
        bool in[PA];
#pragma unroll
        for (int k = 0; k < PA; ++k) {
            const int p = p0 + k * THREADS;
            const int r = p / IW, c = p - r * IW;
            size_t m = 0;
            in[k] = p < NA;
            if (inside) {
                m = (size_t)((y0 - 1 + r) * f.pitch + x0 - 2 + c);
            } else if (in[k]) {
                const int rr = resolve_index(y0 - 1 + r, f.ny, f.edge[2], f.edge[3], 2, fl[k]);
                const int cc = resolve_index(x0 - 2 + c, f.nx, f.edge[0], f.edge[1], 1, fl[k]);
                if (rr >= 0 && cc >= 0)
                    m = (size_t)rr * f.pitch + cc;
                else
                    in[k] = false;  // behind a bounce-back edge: unusable
            }
            if (in[k]) {  // solid nodes are loaded too and dropped below
                ty[k] = f.type[m];
                Dn[k] = f.D[m];
#pragma unroll
                for (int b = 0; b < 9; ++b) g[k][b] = gin[b * plane + m];
            }
        }
#pragma unroll
        for (int k = 0; k < PA; ++k) {
            const int p = p0 + k * THREADS;
            if (p >= NA) continue;
            const int r = p / IW, c = p - r * IW;
            const bool ok = in[k] && (ty[k] & KIND_MASK) != K_SOLID;
            sm.use[r][c] = ok ? 1 : 0;
            all_use &= ok ? 1 : 0;
            if (!ok) continue;
            const T D = Dn[k];
            T eta, mx, my;
            elab_moments(g[k], eta, mx, my);
            const T inv = O::rcp(D + eta);
            const T u = K.e * mx * inv, v = K.e * my * inv;
            T o[9], Fx, Fy;
            elab_equilibrium<T, FM>(K, eta, D, u, v, o, Fx, Fy);
            const T fxs = K.KF * Fx, fys = K.KF * Fy;
            T post[9];
            post[0] = g[k][0] + omega * (o[0] - g[k][0]);
#pragma unroll
            for (int b = 1; b < 9; ++b)
                post[b] = g[k][b] + omega * (o[b] - g[k][b]) + ((b & 1) ? T(1) : T(0.25)) * lat_dot(b, fxs, fys);
            const uint8_t m8 = fl[k];
            if (m8 == 0) {
#pragma unroll
                for (int b = 0; b < 9; ++b) sm.gs[b][r][c] = post[b];
            } else {  // specular ghost: its g*_b serves the mirrored direction
#pragma unroll
                for (int b = 0; b < 9; ++b) sm.gs[mirror_of(b, m8)][r][c] = post[b];
            }
            sm.ed[r][c] = V2{eta, D};
            sm.F[r][c] = V2{fxs, fys};  // read by the node itself only (receivers lie in the grid)
        }
    }
    // a tile whose whole window is usable streams without per-link checks
    const bool dense = __syncthreads_and(all_use) != 0;
    // ---- phase B: stream into the tile's nodes
    for (int q = threadIdx.x; q < TX * TY; q += THREADS) {
        const int qr = q / TX, qc = q % TX;
        const int r = 1 + qr, c = 2 + qc;
        const int x = x0 + qc, y = y0 + qr;
        if (!inside && (x >= f.nx || y >= f.ny)) continue;
        if (!dense && !sm.use[r][c]) continue;
        const V2 me = sm.ed[r][c], Fm = sm.F[r][c];
        T gn[9];
        gn[0] = sm.gs[0][r][c];
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const int cx = lat_cx(a), cy = lat_cy(a);
            const int pr = r - cy, pc = c - cx;
            const T lam = (a & 1) ? T(1) : T(0.25);
            const T frc = lat_dot(a, Fm.x, Fm.y);  // receiver half of KF c_a . (F_x + F_y)
            if (dense || sm.use[pr][pc]) {
                const V2 ep = sm.ed[pr][pc];
                const T bed = -K.G6 * (me.x + ep.x) * (ep.y - me.y);
                gn[a] = sm.gs[a][pr][pc] + lam * (bed + frc);
            } else {
                gn[a] = sm.gs[((a + 3) & 7) + 1][r][c] + lam * frc;
            }
        }
        T eta, mx, my;
        elab_moments(gn, eta, mx, my);
        const size_t idx = inside ? (size_t)(y * f.pitch + x) : (size_t)y * f.pitch + x;
#pragma unroll
        for (int a = 0; a < 9; ++a) gout[a * plane + idx] = gn[a];
        const T inv = O::rcp(me.y + eta);
        f.eta1[idx] = eta;
        f.u1[idx] = K.e * mx * inv;
        f.v1[idx] = K.e * my * inv;
    }
}

// g = o(eta, u, v) at every non-solid node (the equilibrium start), 0 at solids
template <typename T>
__global__ void elab_init_kernel(const T* eta, const T* u, const T* v, const T* D, const uint8_t* type, int nx, int ny,
                                 int pitch, Coef<T> c, T* g, size_t plane)
{
    const size_t n = (size_t)ny * pitch;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % pitch);
        T o[9], Fx, Fy;
        const bool live = x < nx && (type[k] & KIND_MASK) != K_SOLID;
        if (live) elab_equilibrium<T, 0>(c, eta[k], D[k], u[k], v[k], o, Fx, Fy);
#pragma unroll
        for (int a = 0; a < 9; ++a) g[a * plane + k] = live ? o[a] : T(0);
    }
}

}  // namespace maclab
