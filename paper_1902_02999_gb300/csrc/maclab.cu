// maclab.cu -- host side of the C ABI declared in include/maclab.h.
//
// Procedure of Section 3 of Zhou, arXiv:1902.02999: (a) initialise depth and
// velocity, (b) e = 6 nu / dx (Eq. mlb-viscosity), dt = dx / e, (c)-(d)
// update depth and velocity by Eqs. Mac.lb.6 / Mac.lb.7, (e) apply the
// boundary conditions and repeat.  Steps (c)-(e) run in the kernels of
// maclab_kernels.cuh; this file validates the problem, lays out device
// memory, classifies nodes, and sequences the launches.
#include "maclab.h"
#include "maclab_kernels.cuh"
#include "maclab_march.cuh"
#include "maclab_elab.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace maclab;

namespace {

thread_local std::string g_last_error;

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct maclab_s {
    maclab_grid grid{};
    maclab_params params{};
    maclab_bc bc{};
    maclab_allocator alloc{};
    bool has_alloc = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int pitch = 0;
    int prec = MACLAB_F32;
    size_t esize = 4;
    double e = 0, dt = 0;
    int64_t n = 0;             // step count of the current state
    bool have_prev = false;    // the other buffer holds the previous state
    int cur = 0;               // which of the two state buffers is current
    std::vector<Buf> bufs;     // everything allocated, for release
    void* eta[2] = {nullptr, nullptr};
    void* u[2] = {nullptr, nullptr};
    void* v[2] = {nullptr, nullptr};
    void* D = nullptr;         // still-water depth in the state precision
    double* D64 = nullptr;     // still-water depth in double
    uint8_t* type = nullptr;
    int* general = nullptr;    // node indices (j * nx + i) of general-link nodes
    int n_general = 0;
    DirNode* dir = nullptr;
    int n_dir = 0;
    double* stage = nullptr;   // 3 * nx * ny doubles for state transfer
    double* partial = nullptr; // residual block partials
    double* red_out = nullptr; // RED_NVAL doubles
    int red_blocks = 0;
    int ncb = 0, nrb = 0, ty = 0;
    int fmode = 0;             // force terms present: F_WIND | F_FRICTION | F_CORIOLIS
    int grid_blocks = 0;       // cap on step-kernel blocks (0 = one warp per strip)
    int kernel = MACLAB_KERNEL_TILE;  // step kernel: tile, warp strip, TMA-staged tile or row march
    march::Geom mgeom{};       // row-march launch: strips, strip blocks, rows and per-block lists
    bool march_dir_fused = false;  // Dirichlet nodes handled inside the row-march kernel
    bool tma_ok = false;       // tensor maps encoded (FP32, 16-byte aligned buffers)
    TmaMaps tma_maps[2];       // per buffer parity of the state being read
    int tma_grid = 0;          // persistent blocks of the TMA-staged kernel
    int* tma_err = nullptr;    // set by the TMA-staged kernel when a wait timed out
    int graph_steps = 64;      // steps per CUDA-graph replay (even; 0 = no graphs)
    bool steady_bc = true;     // no boundary value depends on time
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // per starting buffer parity
    bool dir_fused = false;    // Dirichlet nodes handled inside the tile kernel
    int* dir_tile_start = nullptr;  // per-tile ranges of the Dirichlet list
    int* gen_tile_start = nullptr;  // per-tile ranges of the bounce-back-link list
    int64_t n_fluid = 0, n_fast = 0;
    double sumD = 0;           // sum of D64 over non-solid nodes
    size_t device_bytes = 0;
    bool profiling = false;
    int64_t prof_steps = 0;    // steps covered by the recorded event pairs
    int tblock = 1;            // temporal blocking: steps per launch of clean tiles
    bool tiles_classified = false;
    int n_clean = 0, n_other = 0;
    int* clean_list = nullptr; // tiles that take two steps per launch
    int* other_list = nullptr; // the rest
    void* mid[3] = {nullptr, nullptr, nullptr};  // scratch state (eta, u, v) at the middle step
    // temporal blocking with the row march: strip blocks taking both steps
    // in one pass (step_march2_kernel), and the others (two single steps
    // through mid, the first with a one-node fringe)
    bool march2_ready = false;
    int n_m2 = 0, n_m2_other = 0;
    int* m2_sel = nullptr;
    int* m2_other = nullptr;
    int graph_end[2] = {0, 1}; // buffer parity after a replay of graph[parity]
    double tau = 1.0;          // relaxation time; != 1: distribution form
    bool newlevel = false;     // hbar at the new time level (per-link kernel for every node)
    int* all_list = nullptr;   // every non-solid node (j * nx + i)
    int n_all = 0;
    bool elab = false;
    void* gdist[2] = {nullptr, nullptr};  // 9 planes of [ny][pitch] per buffer
    void* snap[3] = {nullptr, nullptr, nullptr};  // marked state (eta, u, v), allocated on first mark
    int64_t mark_n = -1;       // step count of the marked state (-1: none)
    std::vector<cudaEvent_t> events;  // pairs around step-kernel launches
    size_t events_used = 0;
    std::string err;
};

namespace {

int fail(maclab_t s, int code, const std::string& msg)
{
    if (s) s->err = msg;
    g_last_error = msg;
    return code;
}

int cuda_fail(maclab_t s, cudaError_t e, const char* what)
{
    return fail(s, MACLAB_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Dirichlet nodes are applied inside the step kernel of this launch shape
bool dirichlet_in_kernel(const maclab_s* s)
{
    if (s->kernel == MACLAB_KERNEL_MARCH) return s->march_dir_fused;
    return s->kernel != MACLAB_KERNEL_STRIP && s->dir_fused;
}

void* dev_alloc(maclab_t s, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (s->has_alloc) {
        p = s->alloc.alloc(bytes, s->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        s->bufs.push_back(Buf{p, bytes});
        s->device_bytes += bytes;
    }
    return p;
}

void release_all(maclab_t s)
{
    for (auto& b : s->bufs) {
        if (s->has_alloc)
            s->alloc.release(b.p, s->alloc.ctx);
        else
            cudaFree(b.p);
    }
    s->bufs.clear();
}

template <typename T>
Coef<T> make_coef(const maclab_params& p, double e, double dt)
{
    const double wmag = std::sqrt(p.wind_u * p.wind_u + p.wind_v * p.wind_v);
    Coef<T> c;
    c.e = (T)e;
    c.G6 = (T)(p.g / (6.0 * e * e));
    c.K6 = (T)(1.0 / (6.0 * e * e));
    c.k3 = (T)(1.0 / (3.0 * e));
    c.k2 = (T)(1.0 / (2.0 * e * e));
    c.k1 = (T)(1.0 / (e * e));
    c.KF = (T)(dt / (6.0 * e));
    c.hdt = (T)(0.5 * dt);
    c.wfx = (T)(p.rho_a * p.Cw * p.wind_u * wmag / p.rho_w);
    c.wfy = (T)(p.rho_a * p.Cw * p.wind_v * wmag / p.rho_w);
    c.Cb = (T)p.Cb;
    c.Om = (T)p.Omega;
    c.nz = (T)-0.0;
    return c;
}

template <typename T>
Fields<T> make_fields(const maclab_s* s)
{
    Fields<T> f;
    const int a = s->cur, b = 1 - s->cur;
    f.eta = (const T*)s->eta[a];
    f.u = (const T*)s->u[a];
    f.v = (const T*)s->v[a];
    f.D = (const T*)s->D;
    f.type = s->type;
    f.eta1 = (T*)s->eta[b];
    f.u1 = (T*)s->u[b];
    f.v1 = (T*)s->v[b];
    f.nx = s->grid.nx;
    f.ny = s->grid.ny;
    f.pitch = s->pitch;
    f.idx32 = (int64_t)s->pitch * s->grid.ny < ((int64_t)1 << 31) ? 1 : 0;
    for (int k = 0; k < 4; ++k) f.edge[k] = s->bc.edge[k];
    f.c = make_coef<T>(s->params, s->e, s->dt);
    return f;
}

// Fields reading the state (ie, iu, iv) and writing (oe, ou, ov)
template <typename T>
Fields<T> fields_io(const maclab_s* s, void* ie, void* iu, void* iv, void* oe, void* ou, void* ov)
{
    Fields<T> f = make_fields<T>(s);
    f.eta = (const T*)ie;
    f.u = (const T*)iu;
    f.v = (const T*)iv;
    f.eta1 = (T*)oe;
    f.u1 = (T*)ou;
    f.v1 = (T*)ov;
    return f;
}

double wave(const maclab_wave& w, double t) { return w.mean + w.amp * std::sin(w.omega * t + w.phase); }

template <typename T>
int launch_step(maclab_t s)
{
    const Fields<T> f = make_fields<T>(s);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (s->profiling) {
        while (s->events.size() < s->events_used + 2) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return cuda_fail(s, cudaGetLastError(), "event");
            s->events.push_back(ev);
        }
        ev0 = s->events[s->events_used];
        ev1 = s->events[s->events_used + 1];
        s->events_used += 2;
        s->prof_steps += 1;
        cudaEventRecord(ev0, s->stream);
    }
    DirValues bv{};
    if (s->n_dir > 0) {
        const double t1 = (double)(s->n + 1) * s->dt;
        for (int k = 0; k < 4; ++k) {
            bv.h[k] = wave(s->bc.h[k], t1);
            bv.qx[k] = wave(s->bc.qx[k], t1);
            bv.qy[k] = wave(s->bc.qy[k], t1);
        }
    }
    const int b = 1 - s->cur;
    if (s->elab) {
        const int tx = (s->grid.nx + tile::TX - 1) / tile::TX, ty = (s->grid.ny + tile::TY - 1) / tile::TY;
        const size_t plane = (size_t)s->pitch * s->grid.ny;
        const size_t smem = sizeof(elab::Smem<T>);
        const T omega = (T)(1.0 / s->tau);
        const dim3 grid(tx, std::min(ty, 65535), (ty + 65534) / 65535);
        switch (s->fmode) {
#define MACLAB_FM(m)                                                                                        \
    case m:                                                                                                 \
        step_elab_kernel<T, m><<<grid, tile::THREADS, smem, s->stream>>>(f, (const T*)s->gdist[s->cur], \
                                                                       (T*)s->gdist[b], plane, omega, ty); \
        break;
            MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
        }
    } else if (s->newlevel) {
        if (s->n_all > 0)
            step_general_kernel<T, true><<<(s->n_all + 127) / 128, 128, 0, s->stream>>>(f, s->all_list, s->n_all);
    } else if (s->kernel == MACLAB_KERNEL_MARCH) {
        // fast nodes, the nodes with a bounce-back link and (when fused) the
        // Dirichlet nodes of every strip block in one launch
        march::Geom g = s->mgeom;
        g.bv = bv;
        if (!s->march_dir_fused) g.dstart = nullptr;
        const int blocks = (g.nitems + march::WARPS - 1) / march::WARPS;
        switch (s->fmode) {
#define MACLAB_FM(m) \
    case m:                                                                                        \
        step_march_kernel<T, m><<<blocks, march::THREADS, march::smem_bytes<T>(), s->stream>>>(f, g); \
        break;
            MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
        }
    } else if (s->kernel != MACLAB_KERNEL_STRIP) {
        // fast nodes, (when fused) Dirichlet nodes and, with the tile kernel,
        // nodes with a bounce-back link in one launch; the TMA-staged kernel
        // leaves the latter to a second launch
        const int tx = (s->grid.nx + tile::TX - 1) / tile::TX, ty = (s->grid.ny + tile::TY - 1) / tile::TY;
        const TileDirichlet td{s->dir_fused ? s->dir_tile_start : nullptr, s->dir, s->D64, bv};
        if constexpr (std::is_same<T, float>::value) {
            if (s->kernel == MACLAB_KERNEL_TMA) {
                const TmaMaps& mp = s->tma_maps[s->cur];
                switch (s->fmode) {
#define MACLAB_FM(m)                                                                                \
    case m:                                                                                         \
        step_tile_tma_kernel<m><<<s->tma_grid, tile::THREADS, tma::SMEM, s->stream>>>(f, mp, tx, tx * ty, td, \
                                                                                   s->tma_err);     \
        break;
                    MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6)
                    MACLAB_FM(7)
#undef MACLAB_FM
                }
            }
        }
        if (s->kernel == MACLAB_KERNEL_TILE) {
            // the tile kernel also updates each tile's nodes with a bounce-back link
            TileDirichlet tg = td;
            tg.gstart = s->gen_tile_start;
            tg.glist = s->general;
            const size_t smem = tile::smem_bytes<T>();
            const dim3 grid(tx, std::min(ty, 65535), (ty + 65534) / 65535);
            switch (s->fmode) {  // compile-time variants for the force terms present
#define MACLAB_FM(m) \
    case m: step_tile_kernel<T, m><<<grid, tile::THREADS, smem, s->stream>>>(f, tx, ty, tg); break;
                MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
            }
        } else if (s->n_general > 0) {
            step_general_kernel<T><<<(s->n_general + 127) / 128, 128, 0, s->stream>>>(f, s->general,
                                                                                      s->n_general);
        }
    } else {
        const int warps = s->ncb * s->nrb;
        int blocks = (warps + WARPS - 1) / WARPS;
        if (s->grid_blocks > 0) blocks = std::min(blocks, s->grid_blocks);
        switch (s->fmode) {
#define MACLAB_FM(m) \
    case m: step_fast_kernel<T, m><<<blocks, 32 * WARPS, 0, s->stream>>>(f, s->ncb, s->nrb, s->ty); break;
            MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
        }
        if (s->n_general > 0)
            step_general_kernel<T><<<(s->n_general + 127) / 128, 128, 0, s->stream>>>(f, s->general,
                                                                                      s->n_general);
    }
    if (s->profiling) cudaEventRecord(ev1, s->stream);
    if (s->n_dir > 0 && !s->elab && (s->newlevel || !dirichlet_in_kernel(s)))
        dirichlet_kernel<T><<<(s->n_dir + 127) / 128, 128, 0, s->stream>>>(
            (T*)s->eta[b], (T*)s->u[b], (T*)s->v[b], (const T*)s->D, s->D64, s->dir, s->n_dir, bv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    s->cur = 1 - s->cur;
    s->n += 1;
    s->have_prev = true;
    return MACLAB_OK;
}

DirValues dir_values(const maclab_s* s, int64_t step)
{
    DirValues bv{};
    if (s->n_dir > 0) {
        const double t1 = (double)step * s->dt;
        for (int k = 0; k < 4; ++k) {
            bv.h[k] = wave(s->bc.h[k], t1);
            bv.qx[k] = wave(s->bc.qx[k], t1);
            bv.qy[k] = wave(s->bc.qy[k], t1);
        }
    }
    return bv;
}

// One single step of the tiles that are not clean, with the bounce-back-link
// and Dirichlet companions, from the state (ie, iu, iv) to (oe, ou, ov).
void other_tiles_step(maclab_t s, void* ie, void* iu, void* iv, void* oe, void* ou, void* ov, int64_t to_step)
{
    const Fields<float> f = fields_io<float>(s, ie, iu, iv, oe, ou, ov);
    const DirValues bv = dir_values(s, to_step);
    const int tx = (s->grid.nx + tile::TX - 1) / tile::TX;
    const TileDirichlet td{s->dir_fused ? s->dir_tile_start : nullptr, s->dir, s->D64, bv, s->gen_tile_start,
                           s->general};
    if (s->n_other > 0) {
        const size_t smem = tile::smem_bytes<float>();
        switch (s->fmode) {
#define MACLAB_FM(m) \
    case m: step_tile_list_kernel<float, m><<<s->n_other, tile::THREADS, smem, s->stream>>>(f, tx, td, s->other_list); break;
            MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
        }
    }
    // the tile-list kernel updates the nodes with a bounce-back link of its
    // tiles (clean tiles have none)
    if (s->n_dir > 0 && !s->dir_fused)
        dirichlet_kernel<float><<<(s->n_dir + 127) / 128, 128, 0, s->stream>>>(
            (float*)oe, (float*)ou, (float*)ov, (const float*)s->D, s->D64, s->dir, s->n_dir, bv);
}

// Two steps with the row march: eligible strip blocks in one pass each
// (step_march2_kernel, state a to state b), the others in two single steps
// through s->mid, the first writing each strip block with its one-node
// fringe so that the second finds every neighbour at the middle state.
void launch_pair_march(maclab_t s, int a, int b)
{
    const size_t smem1 = march::smem_bytes<float>(), smem2 = march::smem2_bytes();
    if (s->n_m2 > 0) {
        const Fields<float> f = fields_io<float>(s, s->eta[a], s->u[a], s->v[a], s->eta[b], s->u[b], s->v[b]);
        const int blocks = (s->n_m2 + march::WARPS - 1) / march::WARPS;
        switch (s->fmode) {
#define MACLAB_FM(m)                                                                                              \
    case m:                                                                                                       \
        step_march2_kernel<m><<<blocks, march::THREADS, smem2, s->stream>>>(f, s->mgeom.items, s->m2_sel, s->n_m2); \
        break;
            MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
        }
    }
    if (s->n_m2_other > 0) {
        const int blocks = (s->n_m2_other + march::WARPS - 1) / march::WARPS;
        march::Geom g1 = s->mgeom, g2 = s->mgeom;
        g1.bv = dir_values(s, s->n + 1);
        g2.bv = dir_values(s, s->n + 2);
        const Fields<float> f1 = fields_io<float>(s, s->eta[a], s->u[a], s->v[a], s->mid[0], s->mid[1], s->mid[2]);
        const Fields<float> f2 = fields_io<float>(s, s->mid[0], s->mid[1], s->mid[2], s->eta[b], s->u[b], s->v[b]);
        switch (s->fmode) {
#define MACLAB_FM(m)                                                                                      \
    case m:                                                                                               \
        step_march_list_kernel<m, true><<<blocks, march::THREADS, smem1, s->stream>>>(f1, g1, s->m2_other,  \
                                                                                   s->n_m2_other);      \
        step_march_list_kernel<m, false><<<blocks, march::THREADS, smem1, s->stream>>>(f2, g2, s->m2_other, \
                                                                                    s->n_m2_other);     \
        break;
            MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
        }
    }
}

// Two steps: clean tiles in one launch (step_tile2_kernel), the other tiles
// in two single steps through the scratch state s->mid (which also receives
// the clean tiles' outer rings at the middle step).  With the row march and
// its strip blocks classified, launch_pair_march instead.
int launch_pair(maclab_t s)
{
    const int a = s->cur, b = 1 - s->cur;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (s->profiling) {
        while (s->events.size() < s->events_used + 2) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return cuda_fail(s, cudaGetLastError(), "event");
            s->events.push_back(ev);
        }
        ev0 = s->events[s->events_used];
        ev1 = s->events[s->events_used + 1];
        s->events_used += 2;
        s->prof_steps += 2;
        cudaEventRecord(ev0, s->stream);
    }
    if (s->kernel == MACLAB_KERNEL_MARCH && s->march2_ready) {
        launch_pair_march(s, a, b);
    } else if (s->n_clean > 0) {
        const Fields<float> f = fields_io<float>(s, s->eta[a], s->u[a], s->v[a], s->mid[0], s->mid[1], s->mid[2]);
        const int tx = (s->grid.nx + tile::TX - 1) / tile::TX;
        const size_t smem = sizeof(tile2::Smem);
        switch (s->fmode) {
#define MACLAB_FM(m)                                                                                             \
    case m:                                                                                                      \
        step_tile2_kernel<m><<<s->n_clean, tile::THREADS, smem, s->stream>>>(f, (float*)s->eta[b], (float*)s->u[b], \
                                                                            (float*)s->v[b], tx, s->clean_list);   \
        break;
            MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
        }
    }
    if (!(s->kernel == MACLAB_KERNEL_MARCH && s->march2_ready)) {
        other_tiles_step(s, s->eta[a], s->u[a], s->v[a], s->mid[0], s->mid[1], s->mid[2], s->n + 1);
        other_tiles_step(s, s->mid[0], s->mid[1], s->mid[2], s->eta[b], s->u[b], s->v[b], s->n + 2);
    }
    if (s->profiling) cudaEventRecord(ev1, s->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "two-step launch");
    s->cur = b;
    s->n += 2;
    s->have_prev = false;  // the middle state is not kept whole
    return MACLAB_OK;
}

// n steps: pairs where temporal blocking is on, the last step always single
int advance(maclab_t s, int64_t n)
{
    const bool pairs_on = s->tblock == 2 && s->prec == MACLAB_F32 && !s->elab && !s->newlevel;
    const int64_t pairs = pairs_on && n >= 3 ? (n - 1) / 2 : 0;
    for (int64_t k = 0; k < pairs; ++k) {
        int rc = launch_pair(s);
        if (rc != MACLAB_OK) return rc;
    }
    for (int64_t k = 2 * pairs; k < n; ++k) {
        int rc = s->prec == MACLAB_F32 ? launch_step<float>(s) : launch_step<double>(s);
        if (rc != MACLAB_OK) return rc;
    }
    return MACLAB_OK;
}

// The residual reduction of the current state against the previous step's
// state, or (since_mark) against the marked state.
template <typename T>
int launch_residual(maclab_t s, bool since_mark = false)
{
    const int a = s->cur, b = 1 - s->cur;
    const void* pe = since_mark ? s->snap[0] : s->eta[b];
    const void* pu = since_mark ? s->snap[1] : s->u[b];
    const void* pv = since_mark ? s->snap[2] : s->v[b];
    residual_partial_kernel<T><<<s->red_blocks, RED_THREADS, 0, s->stream>>>(
        (const T*)pe, (const T*)pu, (const T*)pv, (const T*)s->eta[a],
        (const T*)s->u[a], (const T*)s->v[a], (const T*)s->D, s->type, s->grid.nx, s->grid.ny,
        s->pitch, s->partial);
    residual_final_kernel<<<1, 32 * RED_NVAL, 0, s->stream>>>(s->partial, s->red_blocks, s->red_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "residual launch");
    return MACLAB_OK;
}

// Tensor maps of the TMA-staged kernel: 2D [ny][pitch] views of eta, u, v
// (both buffers), D and the types; boxes of 72 floats / 96 bytes by 18 rows
// (a tile and its halo).  Reads past the grid fill zeros, which only land in
// staged columns the kernel does not use.  Returns false (and leaves the
// TMA kernel off) when the driver entry point is missing, a buffer is not
// 16-byte aligned or an encode fails.
bool encode_tma_maps(maclab_t s)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        cudaGetLastError();
    });
    if (!encode || s->prec != MACLAB_F32) return false;
    auto make = [&](CUtensorMap* m, void* base, CUtensorMapDataType dt, size_t esize, uint32_t box_x) {
        if (((uintptr_t)base & 15) != 0) return false;
        const cuuint64_t dims[2] = {(cuuint64_t)s->grid.nx, (cuuint64_t)s->grid.ny};
        const cuuint64_t strides[1] = {(cuuint64_t)s->pitch * esize};
        const cuuint32_t box[2] = {box_x, (cuuint32_t)tile::IR};
        const cuuint32_t estr[2] = {1, 1};
        return encode(m, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    bool ok = true;
    for (int a = 0; a < 2 && ok; ++a) {
        TmaMaps& m = s->tma_maps[a];
        ok = make(&m.eta, s->eta[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, tma::SRW) &&
             make(&m.u, s->u[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, tma::SRW) &&
             make(&m.v, s->v[a], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, tma::SRW) &&
             make(&m.D, s->D, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, tma::SRW) &&
             make(&m.type, s->type, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, tma::STW);
    }
    return ok;
}

// Nonzero when a TMA-staged step gave up waiting for a copy.
int check_tma_err(maclab_t s)
{
    if (!s->tma_err) return MACLAB_OK;
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, s->tma_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "step status");
    if (flag) return fail(s, MACLAB_E_CUDA, "TMA-staged step: a tensor copy did not arrive in time");
    return MACLAB_OK;
}

int grid_blocks(size_t total, int threads, int cap)
{
    size_t b = (total + threads - 1) / threads;
    return (int)std::max<size_t>(1, std::min<size_t>(b, (size_t)cap));
}

// Distribution form: restart the distributions at the equilibrium of the
// current macroscopic state (buffer s->cur).
int elab_restart(maclab_t s)
{
    const size_t plane = (size_t)s->pitch * s->grid.ny;
    const int a = s->cur;
    if (s->prec == MACLAB_F32)
        elab_init_kernel<float><<<grid_blocks(plane, 256, 4096), 256, 0, s->stream>>>(
            (const float*)s->eta[a], (const float*)s->u[a], (const float*)s->v[a], (const float*)s->D, s->type,
            s->grid.nx, s->grid.ny, s->pitch, make_coef<float>(s->params, s->e, s->dt), (float*)s->gdist[a], plane);
    else
        elab_init_kernel<double><<<grid_blocks(plane, 256, 4096), 256, 0, s->stream>>>(
            (const double*)s->eta[a], (const double*)s->u[a], (const double*)s->v[a], (const double*)s->D, s->type,
            s->grid.nx, s->grid.ny, s->pitch, make_coef<double>(s->params, s->e, s->dt), (double*)s->gdist[a], plane);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "distribution restart");
    return MACLAB_OK;
}

// The device address of host memory the GPU can load and store directly
// (page-locked and mapped into the unified address space: cudaHostAlloc,
// cudaHostRegister), else null (pageable memory takes the staged copies).
void* mapped_host(const void* p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

template <typename T>
int upload_state(maclab_t s, const double* h, const double* u, const double* v)
{
    const size_t N = (size_t)s->grid.nx * s->grid.ny;
    cudaError_t e;
    // pinned, mapped host arrays: the conversion kernel loads them itself
    // (over the host link, no staging copy); otherwise copy to the stage
    const double* dh = (const double*)mapped_host(h);
    const double* du = (const double*)mapped_host(u);
    const double* dv = (const double*)mapped_host(v);
    if (!dh || !du || !dv) {
        if ((e = cudaMemcpyAsync(s->stage, h, N * 8, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(s->stage + N, u, N * 8, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(s->stage + 2 * N, v, N * 8, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
            return cuda_fail(s, e, "state upload");
        dh = s->stage;
        du = s->stage + N;
        dv = s->stage + 2 * N;
    }
    const int a = s->cur, b = 1 - s->cur;
    state_in_kernel<T><<<grid_blocks(N, 256, 4096), 256, 0, s->stream>>>(
        dh, du, dv, s->D64, s->type, (T*)s->eta[a], (T*)s->u[a],
        (T*)s->v[a], (T*)s->eta[b], (T*)s->u[b], (T*)s->v[b], s->grid.nx, s->grid.ny, s->pitch);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(s, e, "state conversion");
    // the host arrays must stay valid until the copies have read them
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(s, e, "state upload");
    s->have_prev = false;
    s->mark_n = -1;  // the marked state belongs to the replaced history
    return MACLAB_OK;
}

template <typename T>
int download_state(maclab_t s, double* h, double* u, double* v)
{
    const size_t N = (size_t)s->grid.nx * s->grid.ny;
    const int a = s->cur;
    // all three arrays pinned and mapped: the conversion kernel stores into
    // them itself; otherwise into the stage, then copies
    double* dh = h ? (double*)mapped_host(h) : nullptr;
    double* du = u ? (double*)mapped_host(u) : nullptr;
    double* dv = v ? (double*)mapped_host(v) : nullptr;
    const bool direct = dh && du && dv;
    state_out_kernel<T><<<grid_blocks(N, 256, 4096), 256, 0, s->stream>>>(
        (const T*)s->eta[a], (const T*)s->u[a], (const T*)s->v[a], s->D64, direct ? dh : s->stage,
        direct ? du : s->stage + N, direct ? dv : s->stage + 2 * N, s->grid.nx, s->grid.ny, s->pitch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "state conversion");
    double* dst[3] = {h, u, v};
    for (int k = 0; k < 3 && !direct; ++k)
        if (dst[k] && (e = cudaMemcpyAsync(dst[k], s->stage + k * N, N * 8, cudaMemcpyDeviceToHost,
                                           s->stream)) != cudaSuccess)
            return cuda_fail(s, e, "state download");
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) return cuda_fail(s, e, "state download");
    return MACLAB_OK;
}

// Rows per warp strip: enough strips to fill every SM a few times over
// while keeping strips tall (each strip re-reads two halo rows).
int choose_tile_rows(int ny, int ncb, int sms)
{
    const int target = sms * 32;  // warps: 32 per SM
    int strips = std::max(1, target / std::max(1, ncb));
    int ty = (ny + strips - 1) / strips;
    ty = std::max(ty, 8);
    ty = std::min(ty, std::max(ny, 1));
    return ty;
}

// Host-side preparation of one grid: validation, node classification,
// Dirichlet list in tile order, still-water depth (procedure steps (a)-(b)
// of Section 3, done once per grid).
struct Prepared {
    int nx = 0, ny = 0, pitch = 0;
    double e = 0, dt = 0;
    maclab_params params{};
    maclab_bc bc{};
    int fmode = 0;
    bool steady_bc = true;
    std::vector<uint8_t> type;      // [ny][pitch], kind | GENERAL_BIT
    std::vector<int> general;       // j * nx + i of nodes with a bounce-back link, in tile order
    std::vector<int> gen_start;     // per-tile ranges of general
    std::vector<DirNode> dirs;      // in tile order, storage indices
    std::vector<int> dir_start;     // per-tile ranges of dirs
    bool dir_fused = false;
    std::vector<double> D64;        // [ny][pitch] still-water depth h_ref - z_b
    double sumD = 0;
    int64_t n_fluid = 0, n_fast = 0;
    int tiles_x = 0, tiles_y = 0;
};

int prepare(const maclab_grid* grid, const maclab_params* params, const maclab_bc* bc, const double* zb,
            const uint8_t* mask, Prepared& P)
{
    if (!grid || !params || !zb || !mask) return fail(nullptr, MACLAB_E_ARG, "grid, params, zb and mask are required");
    const int nx = grid->nx, ny = grid->ny;
    if (nx < 1 || ny < 1) return fail(nullptr, MACLAB_E_ARG, "nx and ny must be >= 1");
    if ((int64_t)nx * ny > (int64_t)1 << 31 || nx > (1 << 30) - 64)
        return fail(nullptr, MACLAB_E_ARG, "grid too large (nx*ny must fit in 31 bits)");
    if (!(grid->dx > 0) || !std::isfinite(grid->dx)) return fail(nullptr, MACLAB_E_ARG, "dx must be > 0");
    if (params->precision != MACLAB_F32 && params->precision != MACLAB_F64)
        return fail(nullptr, MACLAB_E_ARG, "unknown precision");
    const double e = params->e > 0 ? params->e : 6.0 * params->nu / grid->dx;
    if (!(e > 0) || !std::isfinite(e)) return fail(nullptr, MACLAB_E_ARG, "need e > 0 or nu > 0");
    if (!(params->g > 0) || !(params->rho_w > 0)) return fail(nullptr, MACLAB_E_ARG, "need g > 0 and rho_w > 0");
    maclab_bc b{};
    if (bc) b = *bc;
    for (int k = 0; k < 4; ++k)
        if (b.edge[k] < MACLAB_BOUNCEBACK || b.edge[k] > MACLAB_PERIODIC)
            return fail(nullptr, MACLAB_E_ARG, "unknown edge kind");
    if ((b.edge[0] == MACLAB_PERIODIC) != (b.edge[1] == MACLAB_PERIODIC) ||
        (b.edge[2] == MACLAB_PERIODIC) != (b.edge[3] == MACLAB_PERIODIC))
        return fail(nullptr, MACLAB_E_ARG, "periodic edges must come in W/E or S/N pairs");
    const size_t N = (size_t)nx * ny;
    for (size_t k = 0; k < N; ++k)
        if (mask[k] > MACLAB_DIR_HU) return fail(nullptr, MACLAB_E_ARG, "unknown node type in mask");

    P.nx = nx;
    P.ny = ny;
    P.pitch = (nx + 63) / 64 * 64;
    P.e = e;
    P.dt = grid->dx / e;
    P.params = *params;
    P.bc = b;
    for (int k = 0; k < 4; ++k)
        if (b.h[k].amp != 0 || b.qx[k].amp != 0 || b.qy[k].amp != 0) P.steady_bc = false;
    P.fmode = ((params->wind_u != 0 || params->wind_v != 0) ? F_WIND : 0) |
              (params->Cb != 0 ? F_FRICTION : 0) | (params->Omega != 0 ? F_CORIOLIS : 0);
    const int pitch = P.pitch;
    auto kind_at = [&](int i, int j) { return mask[(size_t)j * nx + i]; };
    auto resolve = [&](int i, int n, int lo, int hi) -> int {
        if (i >= 0 && i < n) return i;
        int kd = i < 0 ? lo : hi;
        if (kd == MACLAB_PERIODIC) return ((i % n) + n) % n;
        if (kd == MACLAB_SPECULAR) {
            i = i < 0 ? -1 - i : 2 * n - 1 - i;
            return (i >= 0 && i < n) ? i : -1;
        }
        return -1;
    };
    static const int CX[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
    static const int CY[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};
    P.type.assign((size_t)pitch * ny, (uint8_t)K_SOLID);
    P.D64.assign((size_t)pitch * ny, 0.0);
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const uint8_t kd = kind_at(i, j);
            uint8_t t = kd;
            P.D64[(size_t)j * pitch + i] = params->h_ref - zb[(size_t)j * nx + i];
            if (kd != MACLAB_SOLID) {
                P.n_fluid++;
                P.sumD += params->h_ref - zb[(size_t)j * nx + i];
                if (kd >= MACLAB_DIR_H) {
                    int di = 0, dj = 0, ed;
                    if (i == 0) { di = 1; ed = 0; }
                    else if (i == nx - 1) { di = -1; ed = 1; }
                    else if (j == 0) { dj = 1; ed = 2; }
                    else if (j == ny - 1) { dj = -1; ed = 3; }
                    else return fail(nullptr, MACLAB_E_ARG, "Dirichlet node not on a grid edge");
                    const int i1 = i + di, j1 = j + dj;
                    if (i1 < 0 || i1 >= nx || j1 < 0 || j1 >= ny || kind_at(i1, j1) == MACLAB_SOLID ||
                        kind_at(i1, j1) >= MACLAB_DIR_H)
                        return fail(nullptr, MACLAB_E_ARG,
                                    "the inward node of a Dirichlet node must be non-solid and not Dirichlet");
                    P.dirs.push_back(DirNode{j * pitch + i, j1 * pitch + i1, (int)kd | (ed << 4)});
                } else {
                    bool gen = false;
                    for (int a = 1; a < 9 && !gen; ++a) {
                        const int si = resolve(i - CX[a], nx, b.edge[0], b.edge[1]);
                        const int sj = resolve(j - CY[a], ny, b.edge[2], b.edge[3]);
                        gen = si < 0 || sj < 0 || kind_at(si, sj) == MACLAB_SOLID;
                    }
                    if (gen) {
                        t |= GENERAL_BIT;
                        P.general.push_back(j * nx + i);
                    } else {
                        P.n_fast++;
                    }
                }
            }
            P.type[(size_t)j * pitch + i] = t;
        }
    }
    // Dirichlet nodes in tile order; the tile kernel applies them itself
    // when every inward node is updated by the fast path of the same tile.
    P.tiles_x = (nx + tile::TX - 1) / tile::TX;
    P.tiles_y = (ny + tile::TY - 1) / tile::TY;
    auto tile_of = [&](int idx) {
        const int j = idx / pitch, i = idx - j * pitch;
        return (j / tile::TY) * P.tiles_x + i / tile::TX;
    };
    std::stable_sort(P.dirs.begin(), P.dirs.end(),
                     [&](const DirNode& a, const DirNode& c) { return tile_of(a.x) < tile_of(c.x); });
    P.dir_start.assign((size_t)P.tiles_x * P.tiles_y + 1, 0);
    bool fused = true;
    for (const DirNode& d : P.dirs) {
        const int j1 = d.n1 / pitch, i1 = d.n1 - j1 * pitch;
        fused = fused && tile_of(d.x) == tile_of(d.n1) && !(P.type[(size_t)j1 * pitch + i1] & GENERAL_BIT);
        P.dir_start[tile_of(d.x) + 1]++;
    }
    for (size_t k = 1; k < P.dir_start.size(); ++k) P.dir_start[k] += P.dir_start[k - 1];
    P.dir_fused = fused && !P.dirs.empty();
    // nodes with a bounce-back link in tile order, with per-tile ranges: the
    // tile kernel updates a tile's own ones after its gather
    auto tile_of_node = [&](int g) { return (g / nx / tile::TY) * P.tiles_x + (g % nx) / tile::TX; };
    std::stable_sort(P.general.begin(), P.general.end(),
                     [&](int a, int c) { return tile_of_node(a) < tile_of_node(c); });
    P.gen_start.assign((size_t)P.tiles_x * P.tiles_y + 1, 0);
    for (int g : P.general) P.gen_start[tile_of_node(g) + 1]++;
    for (size_t k = 1; k < P.gen_start.size(); ++k) P.gen_start[k] += P.gen_start[k - 1];
    return MACLAB_OK;
}

// Launch geometry and per-strip-block lists of the row-march kernel.  The
// strip blocks are sized so that all of them are resident at once (one
// wave): strips = nx / 62 + 1 across, rows per block chosen so that
// strips x blocks fills the resident warps of the device.
template <typename T>
int march_blocks_per_sm(int fmode, int* nb)
{
    cudaError_t e = cudaErrorInvalidValue;
    const int smem = (int)march::smem_bytes<T>();
    switch (fmode) {
#define MACLAB_FM(m)                                                                                           \
    case m:                                                                                                    \
        e = cudaFuncSetAttribute(step_march_kernel<T, m>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
        if (e == cudaSuccess)                                                                                  \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, step_march_kernel<T, m>, march::THREADS, smem); \
        break;
        MACLAB_FM(0) MACLAB_FM(1) MACLAB_FM(2) MACLAB_FM(3) MACLAB_FM(4) MACLAB_FM(5) MACLAB_FM(6) MACLAB_FM(7)
#undef MACLAB_FM
    }
    return e == cudaSuccess ? MACLAB_OK : MACLAB_E_CUDA;
}

int setup_march(maclab_t s, const Prepared& P, int sms)
{
    const int nx = P.nx, ny = P.ny, pitch = P.pitch;
    int nb = 0;
    const int rc = s->prec == MACLAB_F32 ? march_blocks_per_sm<float>(s->fmode, &nb)
                                         : march_blocks_per_sm<double>(s->fmode, &nb);
    if (rc != MACLAB_OK) {
        cudaGetLastError();
        return fail(nullptr, MACLAB_E_CUDA, "occupancy of the row-march kernel");
    }
    const int R = std::max(1, nb) * march::WARPS * sms;  // resident warps: one wave
    march::Geom& g = s->mgeom;
    const int S = march::strips(nx);
    g.strips = S;
    // strip blocks (strip, j0, j1) in launch order; blocks are dispatched in
    // index order as warp slots free up
    std::vector<int> it;
    auto add = [&](int st, int j0, int j1) {
        it.push_back(st);
        it.push_back(j0);
        it.push_back(j1);
        it.push_back(0);
    };
    const double phi = MACLAB_MARCH_GUIDED_PHI;
    if (phi > 0) {
        // guided: tall blocks first (one wave), then shorter ones
        const int H1 = std::min(ny, std::max(march::MIN_ROWS, (int)(phi * S * (double)ny / R)));
        const int H2 = std::max(march::MIN_ROWS, H1 / MACLAB_MARCH_GUIDED_DIV);
        std::vector<int> nbig(S);
        int maxbig = 0;
        for (int st = 0; st < S; ++st) {
            nbig[st] = std::min(ny / H1, R / S + (st < R % S ? 1 : 0));
            maxbig = std::max(maxbig, nbig[st]);
        }
        for (int k = 0; k < maxbig; ++k)
            for (int st = 0; st < S; ++st)
                if (k < nbig[st]) add(st, k * H1, (k + 1) * H1);
        std::vector<std::vector<int>> smallb(S);
        size_t maxsmall = 0;
        for (int st = 0; st < S; ++st) {
            const int j0 = nbig[st] * H1, rem = ny - j0;
            if (rem <= 0) continue;
            const int n = (rem + H2 - 1) / H2;
            for (int k = 0; k <= n; ++k) smallb[st].push_back(j0 + (int)((int64_t)k * rem / n));
            maxsmall = std::max(maxsmall, smallb[st].size() - 1);
        }
        for (size_t k = 0; k < maxsmall; ++k)
            for (int st = 0; st < S; ++st)
                if (k + 1 < smallb[st].size()) add(st, smallb[st][k], smallb[st][k + 1]);
    } else {
        // uniform: WAVES strip blocks per resident warp
        const int want = std::max(1, R * march::WAVES / S);
        const int rows = std::min(ny, std::max(march::MIN_ROWS, (ny + want - 1) / want));
        for (int j0 = 0; j0 < ny; j0 += rows)
            for (int st = 0; st < S; ++st) add(st, j0, std::min(ny, j0 + rows));
    }
    const int items = (int)(it.size() / 4);
    g.nitems = items;
    // strip block of each node: per strip, the block index of each row
    std::vector<int> item_of_row((size_t)S * ny, -1);
    for (int t = 0; t < items; ++t)
        for (int j = it[4 * t + 1]; j < it[4 * t + 2]; ++j) item_of_row[(size_t)it[4 * t] * ny + j] = t;
    // plain interior blocks: every row they read and write lies inside the
    // grid (32-bit offsets), and every node they write is a fluid or
    // Dirichlet node without a bounce-back link (no node type is needed)
    const bool idx32 = (int64_t)pitch * ny < ((int64_t)1 << 31);
    for (int t = 0; t < items; ++t) {
        const int st = it[4 * t], j0 = it[4 * t + 1], j1 = it[4 * t + 2], x0 = march::first_col(st);
        bool plain = idx32 && x0 >= 0 && x0 + 64 <= nx && j0 >= 1 && j1 + 1 <= ny;
        for (int j = j0; j < j1 && plain; ++j)
            for (int i = x0 + 1 + march::HALF; i <= x0 + 62 - march::HALF && plain; ++i) {
                const uint8_t ty = P.type[(size_t)j * pitch + i];
                plain = ty == MACLAB_FLUID || ty == MACLAB_DIR_H || ty == MACLAB_DIR_Q || ty == MACLAB_DIR_HU;
            }
        it[4 * t + 3] = plain ? 1 : 0;
    }
    auto item_of = [&](int i, int j) { return item_of_row[(size_t)march::strip_of(i) * ny + j]; };
    // nodes with a bounce-back link, by strip block
    std::vector<int> gl(P.general);
    std::stable_sort(gl.begin(), gl.end(),
                     [&](int a, int c) { return item_of(a % nx, a / nx) < item_of(c % nx, c / nx); });
    std::vector<int> gs((size_t)items + 1, 0);
    for (int n : gl) gs[item_of(n % nx, n / nx) + 1]++;
    for (size_t k = 1; k < gs.size(); ++k) gs[k] += gs[k - 1];
    // Dirichlet nodes, by strip block; fused when each inward node is written
    // by the same strip block's row pass
    std::vector<DirNode> dl(P.dirs);
    auto item_of_idx = [&](int idx) { return item_of(idx % pitch, idx / pitch); };
    std::stable_sort(dl.begin(), dl.end(),
                     [&](const DirNode& a, const DirNode& c) { return item_of_idx(a.x) < item_of_idx(c.x); });
    std::vector<int> ds((size_t)items + 1, 0);
    bool fused = !dl.empty();
    for (const DirNode& d : dl) {
        fused = fused && item_of_idx(d.x) == item_of_idx(d.n1) && !(P.type[d.n1] & GENERAL_BIT);
        ds[item_of_idx(d.x) + 1]++;
    }
    for (size_t k = 1; k < ds.size(); ++k) ds[k] += ds[k - 1];
    s->march_dir_fused = fused;
    int *dgs = nullptr, *dgl = nullptr, *dds = nullptr, *dit = nullptr;
    DirNode* ddl = nullptr;
    bool ok = (dit = (int*)dev_alloc(s, it.size() * sizeof(int))) != nullptr;  // 256-byte aligned (int4 reads)
    if (ok && !gl.empty())
        ok = (dgs = (int*)dev_alloc(s, gs.size() * sizeof(int))) && (dgl = (int*)dev_alloc(s, gl.size() * sizeof(int)));
    if (ok && fused)
        ok = (dds = (int*)dev_alloc(s, ds.size() * sizeof(int))) &&
             (ddl = (DirNode*)dev_alloc(s, dl.size() * sizeof(DirNode)));
    if (!ok) return fail(nullptr, MACLAB_E_NOMEM, "device allocation failed");
    cudaError_t ce = cudaSuccess;
    auto put = [&](void* dst, const void* src, size_t bytes) {
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream);
    };
    put(dit, it.data(), it.size() * sizeof(int));
    if (dgs) {
        put(dgs, gs.data(), gs.size() * sizeof(int));
        put(dgl, gl.data(), gl.size() * sizeof(int));
    }
    if (dds) {
        put(dds, ds.data(), ds.size() * sizeof(int));
        put(ddl, dl.data(), dl.size() * sizeof(DirNode));
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
    if (ce != cudaSuccess) return cuda_fail(nullptr, ce, "upload");
    g.items = dit;
    g.gstart = dgs;
    g.glist = dgl;
    g.dstart = dds;
    g.dlist = ddl;
    g.D64 = s->D64;
    return MACLAB_OK;
}

}  // namespace

extern "C" {

int maclab_abi_version(void) { return MACLAB_ABI_VERSION; }

}  // extern "C"

// Thread-local message for maclab_last_error(NULL), set by other
// translation units of the library.
void maclab_note_error(const std::string& msg) { g_last_error = msg; }

extern "C" {

const char* maclab_last_error(maclab_t sim)
{
    if (sim) return sim->err.c_str();
    return g_last_error.c_str();
}

int maclab_create(const maclab_grid* grid, const maclab_params* params, const maclab_bc* bc,
                  const double* zb, const uint8_t* mask, const double* h0, const double* u0,
                  const double* v0, const maclab_allocator* alloc, void* stream, maclab_t* out)
{
    if (!out) return fail(nullptr, MACLAB_E_ARG, "out is NULL");
    *out = nullptr;
    if ((h0 == nullptr) != (u0 == nullptr) || (h0 == nullptr) != (v0 == nullptr))
        return fail(nullptr, MACLAB_E_ARG, "h0, u0, v0 must be all given or all NULL");
    if (alloc && (!alloc->alloc || !alloc->release))
        return fail(nullptr, MACLAB_E_ARG, "allocator needs alloc and release");
    Prepared P;
    int prc = prepare(grid, params, bc, zb, mask, P);
    if (prc != MACLAB_OK) return prc;
    const int nx = P.nx, ny = P.ny;
    const size_t N = (size_t)nx * ny;

    maclab_s* s = new maclab_s();
    s->grid = *grid;
    s->params = *params;
    s->bc = P.bc;
    s->prec = params->precision;
    s->esize = s->prec == MACLAB_F32 ? 4 : 8;
    // FP32: the row-march kernel (fastest measured on GB300); FP64: tiles
    s->kernel = s->prec == MACLAB_F32 ? MACLAB_KERNEL_MARCH : MACLAB_KERNEL_TILE;
    s->e = P.e;
    s->dt = P.dt;
    s->stream = (cudaStream_t)stream;
    if (alloc) {
        s->alloc = *alloc;
        s->has_alloc = true;
    }
    s->pitch = P.pitch;
    s->steady_bc = P.steady_bc;
    s->fmode = P.fmode;
    cudaGetDevice(&s->device);
    const int pitch = s->pitch;
    s->n_fluid = P.n_fluid;
    s->n_fast = P.n_fast;
    s->sumD = P.sumD;
    s->dir_fused = P.dir_fused;
    std::vector<uint8_t>& type = P.type;
    std::vector<int>& general = P.general;
    std::vector<DirNode>& dirs = P.dirs;
    std::vector<int>& dir_start = P.dir_start;

    // ---- device buffers ----
    const size_t NP = (size_t)pitch * ny;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (sms <= 0) sms = 152;
    s->red_blocks = std::max(1, std::min(sms * 4, (int)((N + RED_THREADS - 1) / RED_THREADS)));
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        ok = (s->eta[k] = dev_alloc(s, NP * s->esize)) && (s->u[k] = dev_alloc(s, NP * s->esize)) &&
             (s->v[k] = dev_alloc(s, NP * s->esize));
    }
    ok = ok && (s->D = dev_alloc(s, NP * s->esize)) && (s->D64 = (double*)dev_alloc(s, NP * 8)) &&
         (s->type = (uint8_t*)dev_alloc(s, NP + 64)) && (s->stage = (double*)dev_alloc(s, 3 * N * 8)) &&
         (s->partial = (double*)dev_alloc(s, (size_t)s->red_blocks * RED_NVAL * 8)) &&
         (s->red_out = (double*)dev_alloc(s, RED_NVAL * 8));
    if (ok && s->prec == MACLAB_F32) ok = (s->tma_err = (int*)dev_alloc(s, sizeof(int))) != nullptr;
    if (ok && !general.empty())
        ok = (s->general = (int*)dev_alloc(s, general.size() * sizeof(int))) &&
             (s->gen_tile_start = (int*)dev_alloc(s, P.gen_start.size() * sizeof(int)));
    if (ok && !dirs.empty()) ok = (s->dir = (DirNode*)dev_alloc(s, dirs.size() * sizeof(DirNode))) != nullptr;
    if (ok && s->dir_fused)
        ok = (s->dir_tile_start = (int*)dev_alloc(s, dir_start.size() * sizeof(int))) != nullptr;
    if (!ok) {
        release_all(s);
        delete s;
        return fail(nullptr, MACLAB_E_NOMEM, "device allocation failed");
    }
    s->n_general = (int)general.size();
    s->n_dir = (int)dirs.size();

    // ---- upload static data ----
    std::vector<double>& D64 = P.D64;
    cudaError_t ce = cudaSuccess;
    auto put = [&](void* dst, const void* src, size_t bytes) {
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream);
    };
    put(s->D64, D64.data(), NP * 8);
    if (s->prec == MACLAB_F32) {
        std::vector<float> Df(NP);
        for (size_t k = 0; k < NP; ++k) Df[k] = (float)D64[k];
        put(s->D, Df.data(), NP * 4);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
    } else {
        put(s->D, D64.data(), NP * 8);
    }
    std::vector<uint8_t> tpad(type);
    tpad.resize(NP + 64, 0);
    put(s->type, tpad.data(), NP + 64);
    if (!general.empty()) {
        put(s->general, general.data(), general.size() * sizeof(int));
        put(s->gen_tile_start, P.gen_start.data(), P.gen_start.size() * sizeof(int));
    }
    if (!dirs.empty()) put(s->dir, dirs.data(), dirs.size() * sizeof(DirNode));
    if (s->dir_fused) put(s->dir_tile_start, dir_start.data(), dir_start.size() * sizeof(int));
    if (s->tma_err && ce == cudaSuccess) ce = cudaMemsetAsync(s->tma_err, 0, sizeof(int), s->stream);
    for (int k = 0; k < 2 && ce == cudaSuccess; ++k) {
        ce = cudaMemsetAsync(s->eta[k], 0, NP * s->esize, s->stream);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(s->u[k], 0, NP * s->esize, s->stream);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(s->v[k], 0, NP * s->esize, s->stream);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->stream);
    if (ce != cudaSuccess) {
        cuda_fail(nullptr, ce, "upload");
        release_all(s);
        delete s;
        return MACLAB_E_CUDA;
    }
    if (h0) {
        int rc = s->prec == MACLAB_F32 ? upload_state<float>(s, h0, u0, v0)
                                        : upload_state<double>(s, h0, u0, v0);
        if (rc != MACLAB_OK) {
            g_last_error = s->err;
            release_all(s);
            delete s;
            return rc;
        }
    }
    // ---- shared memory of the tile kernel (above the 48 KB default for FP64) ----
    {
#ifdef MACLAB_STRIP_KERNEL
        s->kernel = MACLAB_KERNEL_STRIP;
#endif
        cudaError_t ae = cudaSuccess;
#define MACLAB_ATTR(T, m)                                                                                  \
    if (ae == cudaSuccess)                                                                                 \
        ae = cudaFuncSetAttribute(step_tile_kernel<T, m>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)tile::smem_bytes<T>());
        if (s->prec == MACLAB_F32) {
            MACLAB_ATTR(float, 0) MACLAB_ATTR(float, 1) MACLAB_ATTR(float, 2) MACLAB_ATTR(float, 3)
            MACLAB_ATTR(float, 4) MACLAB_ATTR(float, 5) MACLAB_ATTR(float, 6) MACLAB_ATTR(float, 7)
        } else {
            MACLAB_ATTR(double, 0) MACLAB_ATTR(double, 1) MACLAB_ATTR(double, 2) MACLAB_ATTR(double, 3)
            MACLAB_ATTR(double, 4) MACLAB_ATTR(double, 5) MACLAB_ATTR(double, 6) MACLAB_ATTR(double, 7)
        }
#undef MACLAB_ATTR
        if (ae == cudaSuccess && s->prec == MACLAB_F32 && encode_tma_maps(s)) {
            // the TMA-staged kernel: opt in to its shared memory, size its persistent grid
            int per_sm = 0;
#define MACLAB_ATTR(m)                                                                                    \
    if (ae == cudaSuccess)                                                                                \
        ae = cudaFuncSetAttribute(step_tile_tma_kernel<m>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)tma::SMEM);
            MACLAB_ATTR(0) MACLAB_ATTR(1) MACLAB_ATTR(2) MACLAB_ATTR(3) MACLAB_ATTR(4) MACLAB_ATTR(5)
            MACLAB_ATTR(6) MACLAB_ATTR(7)
#undef MACLAB_ATTR
            if (ae == cudaSuccess)
                ae = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_tile_tma_kernel<7>, tile::THREADS,
                                                                   tma::SMEM);
            const int ntiles = P.tiles_x * P.tiles_y;
            if (ae == cudaSuccess && per_sm > 0) {
                s->tma_ok = true;
                s->tma_grid = std::max(1, std::min(ntiles, per_sm * sms));
            }
        }
        if (ae != cudaSuccess) {
            cuda_fail(nullptr, ae, "cudaFuncSetAttribute");
            release_all(s);
            delete s;
            return MACLAB_E_CUDA;
        }
    }
    // ---- launch geometry of the strip kernel ----
    {
        const int cpl = s->prec == MACLAB_F32 ? Cfg<float>::CPL : Cfg<double>::CPL;
        const int w = s->prec == MACLAB_F32 ? strip_width<float>() : strip_width<double>();
        s->ncb = (nx - 1 + cpl + w - 1) / w;
    }
    s->ty = choose_tile_rows(ny, s->ncb, sms);
    s->nrb = (ny + s->ty - 1) / s->ty;
    {
        const int mrc = setup_march(s, P, sms);
        if (mrc != MACLAB_OK) {
            release_all(s);
            delete s;
            return mrc;
        }
    }
    *out = s;
    return MACLAB_OK;
}

int maclab_set_stream(maclab_t s, void* stream)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    s->stream = (cudaStream_t)stream;
    return MACLAB_OK;
}

}  // extern "C"

namespace {

void drop_graphs(maclab_t s)
{
    for (int k = 0; k < 2; ++k) {
        if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
        s->graph[k] = nullptr;
    }
}

// Capture graph_steps launches of the step starting from buffer parity
// s->cur on a private stream (nothing runs), then restore the handle.
int capture_graph(maclab_t s)
{
    cudaError_t e = cudaSuccess;
    if (!s->capture_stream) e = cudaStreamCreateWithFlags(&s->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(s, e, "capture stream");
    const cudaStream_t user = s->stream;
    const int cur = s->cur;
    const int64_t n = s->n;
    const bool have_prev = s->have_prev;
    s->stream = s->capture_stream;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s->capture_stream, cudaStreamCaptureModeThreadLocal);
    int rc = MACLAB_OK;
    if (e == cudaSuccess) {
        rc = advance(s, s->graph_steps);
        e = cudaStreamEndCapture(s->capture_stream, &g);
    }
    s->graph_end[cur] = s->cur;
    s->stream = user;
    s->cur = cur;
    s->n = n;
    s->have_prev = have_prev;
    if (rc != MACLAB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->graph[cur], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->graph[cur] = nullptr;
        return cuda_fail(s, e, "graph capture");
    }
    return MACLAB_OK;
}

}  // namespace

extern "C" {

int maclab_step(maclab_t s, int64_t n)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (n < 0) return fail(s, MACLAB_E_ARG, "n must be >= 0");
    // whole blocks of graph_steps steps replay a captured CUDA graph when the
    // launches do not change from step to step (steady boundary data)
    const bool graphs = s->graph_steps > 0 && s->steady_bc && !s->profiling;
    while (graphs && n >= s->graph_steps) {
        if (!s->graph[s->cur]) {
            int rc = capture_graph(s);
            if (rc != MACLAB_OK) return rc;
        }
        cudaError_t e = cudaGraphLaunch(s->graph[s->cur], s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "graph launch");
        s->n += s->graph_steps;
        s->cur = s->graph_end[s->cur];  // the buffer the captured steps ended in
        s->have_prev = true;            // a graph ends with a single step
        n -= s->graph_steps;
    }
    return advance(s, n);
}

}  // extern "C"

namespace {
// step kernel of an autotune candidate
int kernel_of_choice(int k)
{
    if (k == 0 || k == 6) return MACLAB_KERNEL_TILE;
    if (k == 5) return MACLAB_KERNEL_TMA;
    if (k == 7 || k == 8) return MACLAB_KERNEL_MARCH;
    return MACLAB_KERNEL_STRIP;
}
}  // namespace

extern "C" {

int maclab_autotune(maclab_t s, int trial_steps, int* choice)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (trial_steps < 2) return fail(s, MACLAB_E_ARG, "trial_steps must be >= 2");
    // keep the state: copies of both buffers, restored at the end
    const size_t bytes = (size_t)s->pitch * s->grid.ny * s->esize;
    void* keep[6] = {};
    void* src[6] = {s->eta[0], s->u[0], s->v[0], s->eta[1], s->u[1], s->v[1]};
    for (int k = 0; k < 6; ++k) {
        keep[k] = dev_alloc(s, bytes);
        if (!keep[k]) return fail(s, MACLAB_E_NOMEM, "autotune scratch");
        cudaMemcpyAsync(keep[k], src[k], bytes, cudaMemcpyDeviceToDevice, s->stream);
    }
    const int cur = s->cur;
    const int64_t n0 = s->n;
    const bool hp = s->have_prev;
    const int kernel0 = s->kernel;
    const int ty0 = s->ty;
    const int prof0 = s->profiling;
    // candidates: 0 = tile kernel; k = 1..4 strip kernel with 4 << k rows;
    // 5 = TMA-staged tile kernel; 6 = tile kernel with two steps per launch
    // on clean tiles (FP32 MacLABSWE steps only); 7 = row-march kernel;
    // 8 = row-march kernel with two steps per pass on plain strip blocks
    // (FP32 MacLABSWE steps only)
    const int rows[5] = {0, 8, 16, 32, 64};
    const bool try_pairs = s->prec == MACLAB_F32 && !s->elab && !s->newlevel;
    const int ncand = 9;
    double best = 1e300;
    int best_k = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    s->profiling = true;  // one launch per step (no graph replay) while timing
    int rc = MACLAB_OK;
    s->tblock = 1;
    for (int k = 0; k < ncand && rc == MACLAB_OK; ++k) {
        if (k == 5 && !s->tma_ok) continue;
        if ((k == 6 || k == 8) && !try_pairs) continue;
        if (k == 7) s->tblock = 1;
        if (k == 8) {
            if ((rc = maclab_set_temporal_block(s, 2)) != MACLAB_OK) break;
            if (!s->march2_ready || s->n_m2 == 0) {
                s->tblock = 1;
                continue;
            }
        }
        if (k == 6) {
            if ((rc = maclab_set_temporal_block(s, 2)) != MACLAB_OK) break;
            if (s->n_clean == 0) {
                s->tblock = 1;
                continue;
            }
        }
        s->kernel = kernel_of_choice(k);
        if (k >= 1 && k <= 4) {
            s->ty = std::min(rows[k], s->grid.ny);
            s->nrb = (s->grid.ny + s->ty - 1) / s->ty;
        }
        rc = maclab_step(s, 2);  // warm-up
        cudaEventRecord(e0, s->stream);
        if (rc == MACLAB_OK) rc = maclab_step(s, trial_steps);
        cudaEventRecord(e1, s->stream);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rc == MACLAB_OK && ms < best) {
            best = ms;
            best_k = k;
        }
    }
    s->events_used = 0;
    s->profiling = prof0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->kernel = kernel_of_choice(best_k);
    s->tblock = best_k == 6 || best_k == 8 ? 2 : 1;
    if (best_k >= 1 && best_k <= 4) {
        s->ty = std::min(rows[best_k], s->grid.ny);
    } else {
        s->ty = ty0;
    }
    s->nrb = (s->grid.ny + s->ty - 1) / s->ty;
    (void)kernel0;
    drop_graphs(s);
    for (int k = 0; k < 6; ++k) cudaMemcpyAsync(src[k], keep[k], bytes, cudaMemcpyDeviceToDevice, s->stream);
    cudaStreamSynchronize(s->stream);
    for (int k = 0; k < 6; ++k) {  // give the scratch back
        for (size_t q = 0; q < s->bufs.size(); ++q) {
            if (s->bufs[q].p == keep[k]) {
                if (s->has_alloc) s->alloc.release(keep[k], s->alloc.ctx);
                else cudaFree(keep[k]);
                s->device_bytes -= s->bufs[q].bytes;
                s->bufs.erase(s->bufs.begin() + q);
                break;
            }
        }
    }
    s->cur = cur;
    s->n = n0;
    s->have_prev = hp;
    if (choice) *choice = best_k;
    return rc;
}

int maclab_set_graph_steps(maclab_t s, int steps)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (steps < 0 || (steps & 1)) return fail(s, MACLAB_E_ARG, "steps must be an even number >= 0");
    drop_graphs(s);
    s->graph_steps = steps;
    return MACLAB_OK;
}

int maclab_get_state(maclab_t s, double* h, double* u, double* v)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    const int rc = check_tma_err(s);
    if (rc != MACLAB_OK) return rc;
    return s->prec == MACLAB_F32 ? download_state<float>(s, h, u, v) : download_state<double>(s, h, u, v);
}

int maclab_set_state(maclab_t s, const double* h, const double* u, const double* v)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (!h || !u || !v) return fail(s, MACLAB_E_ARG, "h, u and v are required");
    const int rc = s->prec == MACLAB_F32 ? upload_state<float>(s, h, u, v) : upload_state<double>(s, h, u, v);
    if (rc != MACLAB_OK || !s->elab) return rc;
    return elab_restart(s);
}

}  // extern "C"

namespace {
// out[0] = ||q - q_prev|| / (interval ||q||) and the mass, speed and
// non-finite count, for the previous step's state or the marked one
int residual_common(maclab_t s, double out[4], bool since_mark)
{
    int rc = check_tma_err(s);
    if (rc != MACLAB_OK) return rc;
    rc = s->prec == MACLAB_F32 ? launch_residual<float>(s, since_mark) : launch_residual<double>(s, since_mark);
    if (rc != MACLAB_OK) return rc;
    double r[RED_NVAL];
    cudaError_t e = cudaMemcpyAsync(r, s->red_out, sizeof(r), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "residual");
    const double interval = since_mark ? (double)(s->n - s->mark_n) : 1.0;
    out[0] = r[1] > 0 ? std::sqrt(r[0]) / std::sqrt(r[1]) / interval : 0.0;
    out[1] = s->sumD + r[2];
    out[2] = std::sqrt(r[3]);
    out[3] = r[4];
    if (r[4] > 0 || !std::isfinite(out[0])) return fail(s, MACLAB_E_UNSTABLE, "non-finite values in the state");
    return MACLAB_OK;
}
}  // namespace

extern "C" {

int maclab_residual(maclab_t s, double out[4])
{
    if (!s || !out) return fail(s, MACLAB_E_ARG, "NULL argument");
    if (!s->have_prev) return fail(s, MACLAB_E_STATE, "no step taken since create / set_state");
    return residual_common(s, out, false);
}

int maclab_mark(maclab_t s)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    const size_t bytes = (size_t)s->pitch * s->grid.ny * s->esize;
    for (int k = 0; k < 3; ++k)
        if (!s->snap[k] && !(s->snap[k] = dev_alloc(s, bytes))) return fail(s, MACLAB_E_NOMEM, "mark: device memory");
    const void* src[3] = {s->eta[s->cur], s->u[s->cur], s->v[s->cur]};
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = cudaMemcpyAsync(s->snap[k], src[k], bytes, cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "mark");
    }
    s->mark_n = s->n;
    return MACLAB_OK;
}

int maclab_residual_since_mark(maclab_t s, double out[4])
{
    if (!s || !out) return fail(s, MACLAB_E_ARG, "NULL argument");
    if (s->mark_n < 0 || s->n <= s->mark_n)
        return fail(s, MACLAB_E_STATE, "no marked state, or no step since the mark");
    return residual_common(s, out, true);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Residual without any device allocation.  The block partials and the final
// sums live in one file-scope device array instead of memory the library
// allocates; it exists on every GPU that loads this library, from load until
// process exit.
namespace {
constexpr int NOALLOC_MAX_BLOCKS = 4096;
constexpr int NOALLOC_NODES_PER_THREAD = 16;
constexpr int64_t NOALLOC_MAX_NODES = (int64_t)NOALLOC_MAX_BLOCKS * RED_THREADS * NOALLOC_NODES_PER_THREAD;
constexpr int NOALLOC_MAX_DEVICES = 64;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_BLOCKS * RED_NVAL + RED_NVAL];
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};
CUcontext g_noalloc_ctx[NOALLOC_MAX_DEVICES] = {};

// The context current on this thread (nullptr when none is, or when the
// driver entry point is missing).
CUcontext current_context()
{
    static PFN_cuCtxGetCurrent_v4000 get = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get = (PFN_cuCtxGetCurrent_v4000)fn;
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    if (get && get(&c) != CUDA_SUCCESS) c = nullptr;
    return c;
}

// Device address of the scratch array on the current device.  The array's
// name in host code is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, with that device current: once per device, and
// again whenever the current context is not the one the address was taken
// in (after cudaDeviceReset the library's module is loaded anew).
int noalloc_scratch(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(nullptr, MACLAB_E_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    const CUcontext ctx = current_context();
    if (!g_noalloc_ptr[dev] || !ctx || ctx != g_noalloc_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_ptr[dev] = (double*)p;
        g_noalloc_ctx[dev] = current_context();  // the lookup made the device's context current
    }
    *out = g_noalloc_ptr[dev];
    return MACLAB_OK;
}

template <typename T>
void launch_noalloc(int nx, int ny, int pitch, const void* e0, const void* u0, const void* v0,
                    const void* e1, const void* u1, const void* v1, const void* D, const uint8_t* type,
                    double* scratch, int blocks, cudaStream_t st)
{
    residual_partial_kernel<T><<<blocks, RED_THREADS, 0, st>>>(
        (const T*)e0, (const T*)u0, (const T*)v0, (const T*)e1, (const T*)u1, (const T*)v1, (const T*)D, type,
        nx, ny, pitch, scratch);
    residual_final_kernel<<<1, 32 * RED_NVAL, 0, st>>>(scratch, blocks,
                                                       scratch + (size_t)NOALLOC_MAX_BLOCKS * RED_NVAL);
}
}  // namespace

extern "C" {

int maclab_residual_noalloc(int precision, int nx, int ny, int pitch, const void* eta_prev,
                            const void* u_prev, const void* v_prev, const void* eta_cur, const void* u_cur,
                            const void* v_cur, const void* D, const uint8_t* type, double sum_D,
                            void* stream, double out[4])
{
    if (precision != MACLAB_F32 && precision != MACLAB_F64) return fail(nullptr, MACLAB_E_ARG, "unknown precision");
    if (nx < 1 || ny < 1 || pitch < nx) return fail(nullptr, MACLAB_E_ARG, "need nx, ny >= 1 and pitch >= nx");
    if (!eta_prev || !u_prev || !v_prev || !eta_cur || !u_cur || !v_cur || !D || !type || !out)
        return fail(nullptr, MACLAB_E_ARG, "NULL argument");
    const int64_t N = (int64_t)nx * ny;
    if (N > NOALLOC_MAX_NODES)
        return fail(nullptr, MACLAB_E_ARG,
                    "grid too large for maclab_residual_noalloc: nx*ny must be <= 16777216 "
                    "(its static scratch holds 4096 block partials)");
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != MACLAB_OK) return rc;
    const int per_block = RED_THREADS * NOALLOC_NODES_PER_THREAD;
    const int blocks = (int)std::max<int64_t>(1, (N + per_block - 1) / per_block);
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == MACLAB_F32)
        launch_noalloc<float>(nx, ny, pitch, eta_prev, u_prev, v_prev, eta_cur, u_cur, v_cur, D, type, scratch,
                              blocks, st);
    else
        launch_noalloc<double>(nx, ny, pitch, eta_prev, u_prev, v_prev, eta_cur, u_cur, v_cur, D, type, scratch,
                               blocks, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "residual_noalloc launch");
    double r[RED_NVAL];
    e = cudaMemcpyAsync(r, scratch + (size_t)NOALLOC_MAX_BLOCKS * RED_NVAL, sizeof(r), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "residual_noalloc");
    out[0] = r[1] > 0 ? std::sqrt(r[0]) / std::sqrt(r[1]) : 0.0;
    out[1] = sum_D + r[2];
    out[2] = std::sqrt(r[3]);
    out[3] = r[4];
    if (r[4] > 0 || !std::isfinite(out[0])) return fail(nullptr, MACLAB_E_UNSTABLE, "non-finite values in the state");
    return MACLAB_OK;
}

int maclab_run_to_steady(maclab_t s, double tol, int64_t max_steps, int check_every,
                         int64_t* steps_done, double* r_final)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (check_every < 1 || max_steps < 0 || !(tol >= 0)) return fail(s, MACLAB_E_ARG, "bad tol / max_steps / check_every");
    int64_t done = 0;
    double r = INFINITY;
    int rc = MACLAB_E_STATE;
    while (done < max_steps) {
        const int64_t k = std::min<int64_t>(check_every, max_steps - done);
        if ((rc = maclab_mark(s)) != MACLAB_OK) break;
        if ((rc = maclab_step(s, k)) != MACLAB_OK) break;
        done += k;
        double out[4];
        rc = maclab_residual_since_mark(s, out);
        r = out[0];
        if (rc != MACLAB_OK) break;
        if (r <= tol) break;
        rc = MACLAB_E_STATE;
    }
    if (steps_done) *steps_done = done;
    if (r_final) *r_final = r;
    if (rc == MACLAB_E_STATE) fail(s, rc, "max_steps reached before the residual fell to tol");
    return rc;
}

int maclab_time(maclab_t s, double* t, int64_t* n)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (t) *t = (double)s->n * s->dt;
    if (n) *n = s->n;
    return MACLAB_OK;
}

int maclab_set_tile_rows(maclab_t s, int rows)
{
    return maclab_set_launch(s, rows, s ? s->grid_blocks : 0);
}

int maclab_set_launch(maclab_t s, int rows, int blocks)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (rows < 1 || blocks < 0) return fail(s, MACLAB_E_ARG, "rows must be >= 1 and blocks >= 0");
    s->ty = std::min(rows, s->grid.ny);
    s->nrb = (s->grid.ny + s->ty - 1) / s->ty;
    s->grid_blocks = blocks;
    drop_graphs(s);
    return MACLAB_OK;
}

int maclab_set_step_kernel(maclab_t s, int kernel)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (kernel != MACLAB_KERNEL_TILE && kernel != MACLAB_KERNEL_STRIP && kernel != MACLAB_KERNEL_TMA &&
        kernel != MACLAB_KERNEL_MARCH)
        return fail(s, MACLAB_E_ARG, "unknown step kernel");
    if (kernel == MACLAB_KERNEL_TMA && !s->tma_ok)
        return fail(s, MACLAB_E_ARG, "the TMA-staged kernel needs an FP32 handle with 16-byte aligned buffers");
    s->kernel = kernel;
    drop_graphs(s);
    return MACLAB_OK;
}

int maclab_set_hbar_level(maclab_t s, int level)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (level != 0 && level != 1) return fail(s, MACLAB_E_ARG, "hbar level must be 0 or 1");
    if (level == 1 && s->elab) return fail(s, MACLAB_E_ARG, "the new-level hbar is not offered in the distribution form");
    if (level == 1 && !s->all_list) {
        const int nx = s->grid.nx, ny = s->grid.ny, pitch = s->pitch;
        std::vector<uint8_t> type((size_t)pitch * ny);
        cudaError_t e = cudaMemcpyAsync(type.data(), s->type, type.size(), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "hbar level setup");
        std::vector<int> all;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                if ((type[(size_t)y * pitch + x] & KIND_MASK) != K_SOLID) all.push_back(y * nx + x);
        if (!all.empty()) {
            if (!(s->all_list = (int*)dev_alloc(s, all.size() * sizeof(int))))
                return fail(s, MACLAB_E_NOMEM, "node list");
            e = cudaMemcpyAsync(s->all_list, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "hbar level setup");
        }
        s->n_all = (int)all.size();
    }
    s->newlevel = level == 1;
    drop_graphs(s);
    return MACLAB_OK;
}

int maclab_set_relaxation(maclab_t s, double tau)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (s->newlevel && tau != 1.0) return fail(s, MACLAB_E_ARG, "the distribution form takes the old-level hbar");
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(s, MACLAB_E_ARG, "tau must be finite and > 0.5");
    if (tau == 1.0) {
        s->tau = 1.0;
        s->elab = false;
        drop_graphs(s);
        return MACLAB_OK;
    }
    const int nx = s->grid.nx, ny = s->grid.ny, pitch = s->pitch;
    const size_t NP = (size_t)pitch * ny;
    std::vector<uint8_t> type(NP);
    cudaError_t e = cudaMemcpyAsync(type.data(), s->type, NP, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "relaxation setup");
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const int kind = type[(size_t)y * pitch + x] & KIND_MASK;
            if (kind != K_SOLID && kind != K_FLUID)
                return fail(s, MACLAB_E_ARG, "the distribution form takes fluid and solid nodes only");
        }
    for (int k = 0; k < 2; ++k)
        if (!s->gdist[k] && !(s->gdist[k] = dev_alloc(s, 9 * NP * s->esize)))
            return fail(s, MACLAB_E_NOMEM, "distribution buffers");
    cudaError_t ae = cudaSuccess;
    const size_t smem = s->prec == MACLAB_F32 ? sizeof(elab::Smem<float>) : sizeof(elab::Smem<double>);
#define MACLAB_ATTR(m)                                                                                        \
    if (ae == cudaSuccess)                                                                                    \
        ae = s->prec == MACLAB_F32                                                                            \
                 ? cudaFuncSetAttribute(step_elab_kernel<float, m>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                        (int)smem)                                                            \
                 : cudaFuncSetAttribute(step_elab_kernel<double, m>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                        (int)smem);
    MACLAB_ATTR(0) MACLAB_ATTR(1) MACLAB_ATTR(2) MACLAB_ATTR(3) MACLAB_ATTR(4) MACLAB_ATTR(5) MACLAB_ATTR(6)
    MACLAB_ATTR(7)
#undef MACLAB_ATTR
    if (ae != cudaSuccess) return cuda_fail(s, ae, "cudaFuncSetAttribute");
    s->tau = tau;
    s->elab = true;
    drop_graphs(s);
    return elab_restart(s);
}

int maclab_set_temporal_block(maclab_t s, int k)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (k < 1 || k > 2) return fail(s, MACLAB_E_ARG, "temporal block must be 1 or 2");
    if (k == 2 && s->prec != MACLAB_F32) return fail(s, MACLAB_E_ARG, "temporal blocking needs an FP32 handle");
    if (k == 2 && !s->tiles_classified) {
        // classify the tiles from the node types on the device
        const int nx = s->grid.nx, ny = s->grid.ny, pitch = s->pitch;
        std::vector<uint8_t> type((size_t)pitch * ny);
        cudaError_t e = cudaMemcpyAsync(type.data(), s->type, type.size(), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "temporal block setup");
        const int tiles_x = (nx + tile::TX - 1) / tile::TX, tiles_y = (ny + tile::TY - 1) / tile::TY;
        std::vector<int> clean, other;
        for (int t = 0; t < tiles_x * tiles_y; ++t) {
            const int x0 = (t % tiles_x) * tile::TX, y0 = (t / tiles_x) * tile::TY;
            bool ok = x0 - 2 >= 0 && y0 - 2 >= 0 && x0 + tile::TX + 2 <= nx && y0 + tile::TY + 2 <= ny;
            for (int y = y0 - 2; ok && y < y0 + tile::TY + 2; ++y)
                for (int x = x0 - 2; ok && x < x0 + tile::TX + 2; ++x) {
                    const uint8_t ty = type[(size_t)y * pitch + x];
                    const int kind = ty & KIND_MASK;
                    ok = (kind == K_FLUID || kind == K_NOSLIP) && !(ty & GENERAL_BIT);
                }
            (ok ? clean : other).push_back(t);
        }
        const size_t NP = (size_t)pitch * ny;
        for (int q = 0; q < 3; ++q)
            if (!(s->mid[q] = dev_alloc(s, NP * sizeof(float)))) return fail(s, MACLAB_E_NOMEM, "temporal block scratch");
        if ((!clean.empty() && !(s->clean_list = (int*)dev_alloc(s, clean.size() * sizeof(int)))) ||
            (!other.empty() && !(s->other_list = (int*)dev_alloc(s, other.size() * sizeof(int)))))
            return fail(s, MACLAB_E_NOMEM, "temporal block lists");
        if (!clean.empty()) e = cudaMemcpyAsync(s->clean_list, clean.data(), clean.size() * sizeof(int),
                                                cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess && !other.empty())
            e = cudaMemcpyAsync(s->other_list, other.data(), other.size() * sizeof(int), cudaMemcpyHostToDevice,
                                s->stream);
        for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaMemsetAsync(s->mid[q], 0, NP * sizeof(float), s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "temporal block setup");
        cudaError_t ae = cudaSuccess;
#define MACLAB_ATTR(m)                                                                                      \
    if (ae == cudaSuccess)                                                                                  \
        ae = cudaFuncSetAttribute(step_tile2_kernel<m>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                  (int)sizeof(tile2::Smem));                                                \
    if (ae == cudaSuccess)                                                                                  \
        ae = cudaFuncSetAttribute(step_tile_list_kernel<float, m>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)tile::smem_bytes<float>());
        MACLAB_ATTR(0) MACLAB_ATTR(1) MACLAB_ATTR(2) MACLAB_ATTR(3) MACLAB_ATTR(4) MACLAB_ATTR(5) MACLAB_ATTR(6)
        MACLAB_ATTR(7)
#undef MACLAB_ATTR
        if (ae != cudaSuccess) return cuda_fail(s, ae, "cudaFuncSetAttribute");
        s->n_clean = (int)clean.size();
        s->n_other = (int)other.size();
        s->tiles_classified = true;
    }
    if (k == 2 && !s->march2_ready && s->mgeom.items && (s->n_dir == 0 || s->march_dir_fused)) {
        // row-march strip blocks: both steps in one pass when rows j0 - 2 ..
        // j1 + 1 and the strip's 64 columns lie inside the grid and hold only
        // fluid nodes (no edge rule, wall, link or Dirichlet node reaches
        // two consecutive steps of the block)
        const int nx = s->grid.nx, ny = s->grid.ny, pitch = s->pitch, nit = s->mgeom.nitems;
        std::vector<uint8_t> type((size_t)pitch * ny);
        std::vector<int> it((size_t)4 * nit);
        cudaError_t e = cudaMemcpyAsync(type.data(), s->type, type.size(), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(it.data(), s->mgeom.items, it.size() * sizeof(int), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "temporal block setup");
        const bool idx32 = (int64_t)pitch * ny < ((int64_t)1 << 31);
        std::vector<int> two, rest;
        for (int t = 0; t < nit; ++t) {
            const int x0 = march::first_col(it[4 * t]), j0 = it[4 * t + 1], j1 = it[4 * t + 2];
            bool ok = idx32 && x0 >= 0 && x0 + 64 <= nx && j0 - 2 >= 0 && j1 + 2 <= ny;
            for (int y = j0 - 2; ok && y <= j1 + 1; ++y)
                for (int x = x0; ok && x < x0 + 64; ++x) ok = type[(size_t)y * pitch + x] == MACLAB_FLUID;
            (ok ? two : rest).push_back(t);
        }
        const size_t NP = (size_t)pitch * ny;
        for (int q = 0; q < 3; ++q)
            if (!s->mid[q]) {
                if (!(s->mid[q] = dev_alloc(s, NP * sizeof(float)))) return fail(s, MACLAB_E_NOMEM, "temporal block scratch");
                if ((e = cudaMemsetAsync(s->mid[q], 0, NP * sizeof(float), s->stream)) != cudaSuccess)
                    return cuda_fail(s, e, "temporal block setup");
            }
        if ((!two.empty() && !(s->m2_sel = (int*)dev_alloc(s, two.size() * sizeof(int)))) ||
            (!rest.empty() && !(s->m2_other = (int*)dev_alloc(s, rest.size() * sizeof(int)))))
            return fail(s, MACLAB_E_NOMEM, "temporal block lists");
        if (!two.empty())
            e = cudaMemcpyAsync(s->m2_sel, two.data(), two.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess && !rest.empty())
            e = cudaMemcpyAsync(s->m2_other, rest.data(), rest.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "temporal block setup");
        cudaError_t ae = cudaSuccess;
#define MACLAB_ATTR(m)                                                                                         \
    if (ae == cudaSuccess)                                                                                     \
        ae = cudaFuncSetAttribute(step_march2_kernel<m>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                  (int)march::smem2_bytes());                                                  \
    if (ae == cudaSuccess)                                                                                     \
        ae = cudaFuncSetAttribute(step_march_list_kernel<m, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)march::smem_bytes<float>());                                            \
    if (ae == cudaSuccess)                                                                                     \
        ae = cudaFuncSetAttribute(step_march_list_kernel<m, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)march::smem_bytes<float>());
        MACLAB_ATTR(0) MACLAB_ATTR(1) MACLAB_ATTR(2) MACLAB_ATTR(3) MACLAB_ATTR(4) MACLAB_ATTR(5) MACLAB_ATTR(6)
        MACLAB_ATTR(7)
#undef MACLAB_ATTR
        if (ae != cudaSuccess) return cuda_fail(s, ae, "cudaFuncSetAttribute");
        s->n_m2 = (int)two.size();
        s->n_m2_other = (int)rest.size();
        s->march2_ready = true;
    }
    s->tblock = k;
    drop_graphs(s);
    return MACLAB_OK;
}

int maclab_set_profiling(maclab_t s, int on)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    s->profiling = on != 0;
    s->events_used = 0;
    s->prof_steps = 0;
    return MACLAB_OK;
}

}  // extern "C"

namespace {
// Eight independent FMA chains per thread (x <- a x + b, |a| < 1, so the
// values stay normal and bounded): the FP64 pipe's throughput, not its
// latency, sets the pace.
__global__ void fp64_rate_kernel(double* sink, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __fma_rn(x[k], a, b);
    }
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += x[k];
    if (t == -1.0) sink[blockIdx.x] = t;  // never true: keeps the chains live
}
}  // namespace

extern "C" {

int maclab_measure_fp64(double* tflops)
{
    if (!tflops) return fail(nullptr, MACLAB_E_ARG, "NULL argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "device query");
    const int threads = 256, blocks = 8 * sms, iters = 4096;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, 0);
        fp64_rate_kernel<<<blocks, threads>>>(nullptr, iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, 0);
        e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, ms);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "FP64 rate kernel");
    const double flops = 2.0 * 8.0 * iters * (double)threads * blocks;  // an FMA is two flops
    *tflops = flops / (best * 1e-3) / 1e12;
    return MACLAB_OK;
}

int maclab_get_profile(maclab_t s, double* ms, int64_t* launches)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "profile");
    double total = 0;
    for (size_t k = 0; k + 1 < s->events_used; k += 2) {
        float t = 0;
        if ((e = cudaEventElapsedTime(&t, s->events[k], s->events[k + 1])) != cudaSuccess)
            return cuda_fail(s, e, "profile");
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = s->prof_steps;
    s->events_used = 0;
    s->prof_steps = 0;
    return MACLAB_OK;
}

int maclab_get_info(maclab_t s, maclab_info* info)
{
    if (!s || !info) return fail(s, MACLAB_E_ARG, "NULL argument");
    info->nx = s->grid.nx;
    info->ny = s->grid.ny;
    info->pitch = s->pitch;
    info->precision = s->prec;
    info->dx = s->grid.dx;
    info->e = s->e;
    info->dt = s->dt;
    info->nu = s->e * s->grid.dx / 6.0;
    info->n_dirichlet = s->n_dir;
    info->n_fluid = s->n_fluid;
    info->n_fast = s->n_fast;
    info->device_bytes = s->device_bytes;
    info->tile_rows = s->ty;
    info->step_kernel = s->kernel;
    info->dirichlet_fused = dirichlet_in_kernel(s) ? 1 : 0;
    info->temporal_block = s->tblock;
    info->two_step_blocks = s->march2_ready ? s->n_m2 : 0;
    info->clean_tiles = s->n_clean;
    info->tau = s->tau;
    info->hbar_level = s->newlevel ? 1 : 0;
    return MACLAB_OK;
}

int maclab_device_state(maclab_t s, void** eta, void** u, void** v)
{
    if (!s) return fail(nullptr, MACLAB_E_ARG, "NULL handle");
    if (eta) *eta = s->eta[s->cur];
    if (u) *u = s->u[s->cur];
    if (v) *v = s->v[s->cur];
    return MACLAB_OK;
}

void maclab_destroy(maclab_t s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    drop_graphs(s);
    if (s->capture_stream) cudaStreamDestroy(s->capture_stream);
    release_all(s);
    delete s;
}

}  // extern "C"

// ===========================================================================
// Batches: many independent grids advanced together (one step-kernel launch
// for all of them over a packed tile list).
struct maclab_batch_s {
    int count = 0;
    int prec = MACLAB_F32;
    size_t esize = 4;
    cudaStream_t stream = nullptr;
    maclab_allocator alloc{};
    bool has_alloc = false;
    std::vector<Buf> bufs;
    size_t device_bytes = 0;
    // per-instance host facts
    std::vector<int> nx, ny, pitch, tiles_x, tile0, ntiles;
    std::vector<size_t> off;        // element offset of the instance in the packed arrays
    std::vector<double> dt, sumD;
    std::vector<int64_t> nodes;
    int total_tiles = 0;
    size_t total_np = 0;
    // device arrays
    void* eta[2] = {nullptr, nullptr};
    void* u[2] = {nullptr, nullptr};
    void* v[2] = {nullptr, nullptr};
    void* D = nullptr;
    double* D64 = nullptr;
    uint8_t* type = nullptr;
    double* stage = nullptr;
    void* insts = nullptr;          // BatchInst<T>[count]
    int* tile_inst = nullptr;
    uint8_t* active = nullptr;
    int2* general = nullptr;        // (instance, j * nx + i) of nodes with a bounce-back link
    int n_general = 0;
    int* gen_nodes = nullptr;       // the same nodes (j * nx + i) in batch-tile order
    int* gen_tile_start = nullptr;  // per batch tile ranges of gen_nodes
    DirNode* dirs = nullptr;
    int* dir_owner = nullptr;
    int* dir_start = nullptr;       // per batch tile, when fused
    int n_dir = 0;
    bool dir_fused = false;
    double* partial = nullptr;
    double* red_out = nullptr;
    std::vector<uint8_t> active_host;
    int cur = 0;
    int64_t n = 0;
    bool have_prev = false;
    int graph_steps = 64;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // persistent steps (one cooperative launch for many steps)
    int persist_mode = 0;           // 0 one launch per step, 1 persistent
    int persist_grid = 0;           // resident blocks of the persistent kernel (0: not available)
    GridBarrier* barrier = nullptr;
    int* persist_err = nullptr;     // set when a grid-barrier wait timed out
    unsigned int bar_extra = 0;     // test hook: arrivals the grid barrier expects beyond the grid
    unsigned int bar_polls = BARRIER_POLLS;  // polls before a grid-barrier wait gives up
    bool broken = false;            // a persistent step stopped early: the state must be reloaded
    std::vector<uint8_t> reloaded;  // instances set since the batch broke
    void* snap[3] = {nullptr, nullptr, nullptr};  // marked state, packed like eta / u / v
    int64_t mark_n = -1;            // step count of the marked state (-1: none)
    std::string err;
};

namespace {

int bfail(maclab_batch_t b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    g_last_error = msg;
    return code;
}

void* bdev_alloc(maclab_batch_t b, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (b->has_alloc) {
        p = b->alloc.alloc(bytes, b->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        b->bufs.push_back(Buf{p, bytes});
        b->device_bytes += bytes;
    }
    return p;
}

void brelease(maclab_batch_t b)
{
    for (int k = 0; k < 2; ++k)
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (auto& x : b->bufs) {
        if (b->has_alloc)
            b->alloc.release(x.p, b->alloc.ctx);
        else
            cudaFree(x.p);
    }
    b->bufs.clear();
}

template <typename T>
void fill_insts(maclab_batch_t b, const std::vector<Prepared>& P, std::vector<BatchInst<T>>& out)
{
    out.resize(b->count);
    for (int i = 0; i < b->count; ++i) {
        BatchInst<T>& in = out[i];
        const size_t o = b->off[i];
        for (int par = 0; par < 2; ++par) {
            Fields<T>& f = in.f[par];
            f.eta = (const T*)b->eta[par] + o;
            f.u = (const T*)b->u[par] + o;
            f.v = (const T*)b->v[par] + o;
            f.eta1 = (T*)b->eta[1 - par] + o;
            f.u1 = (T*)b->u[1 - par] + o;
            f.v1 = (T*)b->v[1 - par] + o;
            f.D = (const T*)b->D + o;
            f.type = b->type + o;
            f.nx = P[i].nx;
            f.ny = P[i].ny;
            f.pitch = P[i].pitch;
            f.idx32 = (int64_t)P[i].pitch * P[i].ny < ((int64_t)1 << 31) ? 1 : 0;
            for (int k = 0; k < 4; ++k) f.edge[k] = P[i].bc.edge[k];
            f.c = make_coef<T>(P[i].params, P[i].e, P[i].dt);
        }
        in.tiles_x = P[i].tiles_x;
        in.tile0 = b->tile0[i];
        in.ntiles = b->ntiles[i];
        in.pad = 0;
        in.D64 = b->D64 + o;
        for (int k = 0; k < 4; ++k) {  // steady boundary data
            in.bv.h[k] = P[i].bc.h[k].mean;
            in.bv.qx[k] = P[i].bc.qx[k].mean;
            in.bv.qy[k] = P[i].bc.qy[k].mean;
        }
    }
}

// Resident blocks of the persistent batch kernel (0 when the device has no
// cooperative launch).
template <typename T>
cudaError_t persistent_setup(maclab_batch_t b)
{
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_batch_persistent_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile::smem_bytes<T>());
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_batch_persistent_kernel<T>, tile::THREADS,
                                                          tile::smem_bytes<T>());
    b->persist_grid = (e == cudaSuccess && coop) ? per_sm * sms : 0;
    return e;
}

// Whether maclab_batch_step takes the persistent kernel (on request only).
bool use_persistent(const maclab_batch_s* b) { return b->persist_grid > 0 && b->persist_mode == 1; }

// n steps in cooperative launches of at most 4096 steps each.
template <typename T>
int batch_persistent(maclab_batch_t b, int64_t n)
{
    const BatchInst<T>* insts = (const BatchInst<T>*)b->insts;
    const int grid = std::min(b->total_tiles, b->persist_grid);
    const unsigned int nbar = (unsigned int)grid + b->bar_extra;
    while (n > 0) {
        int k = (int)std::min<int64_t>(n, 4096);
        int par = b->cur;
        const int* dstart = b->dir_fused ? b->dir_start : nullptr;
        int nsep = b->dir_fused ? 0 : b->n_dir;
        unsigned int gen0 = 0;
        void* args[] = {(void*)&insts, (void*)&b->tile_inst, (void*)&b->total_tiles, (void*)&b->active,
                        (void*)&par, (void*)&k, (void*)&dstart, (void*)&b->dirs, (void*)&b->general,
                        (void*)&b->n_general, (void*)&b->dir_owner, (void*)&nsep, (void*)&b->barrier,
                        (void*)&gen0, (void*)&b->persist_err, (void*)&nbar, (void*)&b->bar_polls};
        cudaError_t e = cudaMemsetAsync(b->barrier, 0, sizeof(GridBarrier), b->stream);
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel((const void*)step_batch_persistent_kernel<T>, dim3(grid),
                                            dim3(tile::THREADS), args, tile::smem_bytes<T>(), b->stream);
        if (e != cudaSuccess)
            return bfail(b, MACLAB_E_CUDA, std::string("persistent batch launch: ") + cudaGetErrorString(e));
        b->cur ^= (k & 1);
        b->n += k;
        b->have_prev = true;
        n -= k;
    }
    return MACLAB_OK;
}

// MACLAB_E_CUDA once a grid-barrier wait of the persistent kernel has timed out.
int check_persist_err(maclab_batch_t b)
{
    if (!b->persist_err || b->broken) return MACLAB_OK;  // a known failure is reported by batch_usable
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, b->persist_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("persistent error flag: ") + cudaGetErrorString(e));
    if (flag) {
        // the blocks left at different steps: the device state matches no
        // step count, so the batch refuses further use until every
        // instance is reloaded
        b->broken = true;
        b->reloaded.assign(b->count, 0);
        return bfail(b, MACLAB_E_CUDA, "a grid-barrier wait of the persistent batch kernel timed out");
    }
    return MACLAB_OK;
}

int batch_usable(maclab_batch_t b)
{
    if (!b->broken) return MACLAB_OK;
    return bfail(b, MACLAB_E_STATE,
                 "a persistent step stopped early; reload every instance (maclab_batch_set_state) to continue");
}

template <typename T>
int batch_launch(maclab_batch_t b, cudaStream_t st)
{
    const int par = b->cur;
    const BatchInst<T>* insts = (const BatchInst<T>*)b->insts;
    // the tiles also update their own nodes with a bounce-back link
    step_batch_kernel<T><<<b->total_tiles, tile::THREADS, tile::smem_bytes<T>(), st>>>(
        insts, b->tile_inst, b->active, par, b->dir_fused ? b->dir_start : nullptr, b->dirs, b->gen_tile_start,
        b->gen_nodes);
    if (b->n_dir > 0 && !b->dir_fused)
        batch_dirichlet_kernel<T><<<(b->n_dir + 127) / 128, 128, 0, st>>>(insts, b->dir_owner, b->dirs,
                                                                           b->n_dir, b->active, par);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("batch step launch: ") + cudaGetErrorString(e));
    b->cur = 1 - b->cur;
    b->n += 1;
    b->have_prev = true;
    return MACLAB_OK;
}

int batch_one(maclab_batch_t b, cudaStream_t st)
{
    return b->prec == MACLAB_F32 ? batch_launch<float>(b, st) : batch_launch<double>(b, st);
}

int batch_capture(maclab_batch_t b)
{
    cudaError_t e = cudaSuccess;
    if (!b->capture_stream) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, "capture stream");
    const int cur = b->cur;
    const int64_t n = b->n;
    const bool hp = b->have_prev;
    cudaGraph_t g = nullptr;
    int rc = MACLAB_OK;
    e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < b->graph_steps && rc == MACLAB_OK; ++k) rc = batch_one(b, b->capture_stream);
        e = cudaStreamEndCapture(b->capture_stream, &g);
    }
    b->cur = cur;
    b->n = n;
    b->have_prev = hp;
    if (rc != MACLAB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[cur], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph[cur] = nullptr;
        return bfail(b, MACLAB_E_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    return MACLAB_OK;
}

template <typename T>
int batch_residual_t(maclab_batch_t b, double* out, bool since_mark = false)
{
    // the state before the last step sits in buffer 1 - cur: parity 1 - cur
    const int par = 1 - b->cur;
    const BatchInst<T>* insts = (const BatchInst<T>*)b->insts;
    const int c = b->cur;
    const T* se = since_mark ? (const T*)b->snap[0] : nullptr;
    batch_residual_tile_kernel<T><<<b->total_tiles, RED_THREADS, 0, b->stream>>>(
        insts, b->tile_inst, par, b->partial, se, (const T*)b->snap[1], (const T*)b->snap[2],
        (const T*)b->eta[c], (const T*)b->u[c], (const T*)b->v[c]);
    batch_residual_final_kernel<T><<<(b->count + 7) / 8, 256, 0, b->stream>>>(insts, b->count, b->partial,
                                                                             b->red_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("batch residual: ") + cudaGetErrorString(e));
    std::vector<double> r((size_t)b->count * RED_NVAL);
    e = cudaMemcpyAsync(r.data(), b->red_out, r.size() * 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("batch residual: ") + cudaGetErrorString(e));
    int rc = MACLAB_OK;
    const double interval = since_mark ? (double)(b->n - b->mark_n) : 1.0;
    for (int i = 0; i < b->count; ++i) {
        const double* q = &r[(size_t)i * RED_NVAL];
        out[4 * i + 0] = q[1] > 0 ? std::sqrt(q[0]) / std::sqrt(q[1]) / interval : 0.0;
        out[4 * i + 1] = b->sumD[i] + q[2];
        out[4 * i + 2] = std::sqrt(q[3]);
        out[4 * i + 3] = q[4];
        if (q[4] > 0 || !std::isfinite(out[4 * i])) rc = MACLAB_E_UNSTABLE;
    }
    if (rc != MACLAB_OK) bfail(b, rc, "non-finite values in a batch instance");
    return rc;
}

// Give an instance the same state in both buffers (so that it stays put
// while inactive, whatever the batch's buffer parity).
int batch_freeze(maclab_batch_t b, int i)
{
    const size_t bytes = (size_t)b->pitch[i] * b->ny[i] * b->esize;
    const size_t o = b->off[i] * b->esize;
    const int c = b->cur, d = 1 - b->cur;
    void* src[3] = {b->eta[c], b->u[c], b->v[c]};
    void* dst[3] = {b->eta[d], b->u[d], b->v[d]};
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = cudaMemcpyAsync((char*)dst[k] + o, (const char*)src[k] + o, bytes, cudaMemcpyDeviceToDevice,
                                        b->stream);
        if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, "batch freeze");
    }
    return MACLAB_OK;
}

}  // namespace

extern "C" {

int maclab_batch_create(int count, const maclab_grid* grids, const maclab_params* params, const maclab_bc* bcs,
                        const double* const* zb, const uint8_t* const* mask, const double* const* h0,
                        const double* const* u0, const double* const* v0, const maclab_allocator* alloc,
                        void* stream, maclab_batch_t* out)
{
    if (!out) return bfail(nullptr, MACLAB_E_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !grids || !params || !zb || !mask) return bfail(nullptr, MACLAB_E_ARG, "bad batch arguments");
    if (alloc && (!alloc->alloc || !alloc->release))
        return bfail(nullptr, MACLAB_E_ARG, "allocator needs alloc and release");
    std::vector<Prepared> P(count);
    for (int i = 0; i < count; ++i) {
        int rc = prepare(&grids[i], &params[i], bcs ? &bcs[i] : nullptr, zb[i], mask[i], P[i]);
        if (rc != MACLAB_OK) return bfail(nullptr, rc, "instance " + std::to_string(i) + ": " + g_last_error);
        if (params[i].precision != params[0].precision)
            return bfail(nullptr, MACLAB_E_ARG, "all instances of a batch need the same precision");
        if (!P[i].steady_bc)
            return bfail(nullptr, MACLAB_E_ARG, "batch instances need time-independent boundary data");
        const bool has0 = h0 && h0[i], has1 = u0 && u0[i], has2 = v0 && v0[i];
        if (has0 != has1 || has0 != has2)
            return bfail(nullptr, MACLAB_E_ARG, "h0, u0, v0 of an instance must be all given or all NULL");
    }
    maclab_batch_s* b = new maclab_batch_s();
    b->count = count;
    b->prec = params[0].precision;
    b->esize = b->prec == MACLAB_F32 ? 4 : 8;
    b->stream = (cudaStream_t)stream;
    if (alloc) {
        b->alloc = *alloc;
        b->has_alloc = true;
    }
    size_t maxN = 0;
    std::vector<int> tile_inst;
    std::vector<int2> general;
    std::vector<DirNode> dirs;
    std::vector<int> dir_owner, dir_start(1, 0);
    std::vector<int> gen_nodes, gen_start(1, 0);   // bounce-back-link nodes per batch tile
    bool fused = true;
    for (int i = 0; i < count; ++i) {
        const Prepared& p = P[i];
        b->nx.push_back(p.nx);
        b->ny.push_back(p.ny);
        b->pitch.push_back(p.pitch);
        b->tiles_x.push_back(p.tiles_x);
        b->tile0.push_back(b->total_tiles);
        b->ntiles.push_back(p.tiles_x * p.tiles_y);
        b->off.push_back(b->total_np);
        b->dt.push_back(p.dt);
        b->sumD.push_back(p.sumD);
        b->nodes.push_back((int64_t)p.nx * p.ny);
        b->total_np += (size_t)p.pitch * p.ny;
        maxN = std::max(maxN, (size_t)p.nx * p.ny);
        for (int t = 0; t < p.tiles_x * p.tiles_y; ++t) {
            tile_inst.push_back(i);
            for (int k = p.dir_start[t]; k < p.dir_start[t + 1]; ++k) {
                dirs.push_back(p.dirs[k]);
                dir_owner.push_back(i);
            }
            dir_start.push_back((int)dirs.size());
            for (int k = p.gen_start[t]; k < p.gen_start[t + 1]; ++k) gen_nodes.push_back(p.general[k]);
            gen_start.push_back((int)gen_nodes.size());
        }
        b->total_tiles += p.tiles_x * p.tiles_y;
        for (int g : p.general) general.push_back(make_int2(i, g));
        fused = fused && (p.dirs.empty() || p.dir_fused);
    }
    b->n_general = (int)general.size();
    b->n_dir = (int)dirs.size();
    b->dir_fused = fused && b->n_dir > 0;
    const size_t NP = b->total_np;
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k)
        ok = (b->eta[k] = bdev_alloc(b, NP * b->esize)) && (b->u[k] = bdev_alloc(b, NP * b->esize)) &&
             (b->v[k] = bdev_alloc(b, NP * b->esize));
    const size_t inst_bytes = b->prec == MACLAB_F32 ? sizeof(BatchInst<float>) : sizeof(BatchInst<double>);
    ok = ok && (b->D = bdev_alloc(b, NP * b->esize)) && (b->D64 = (double*)bdev_alloc(b, NP * 8)) &&
         (b->type = (uint8_t*)bdev_alloc(b, NP + 64)) && (b->stage = (double*)bdev_alloc(b, 3 * maxN * 8)) &&
         (b->insts = bdev_alloc(b, inst_bytes * count)) &&
         (b->tile_inst = (int*)bdev_alloc(b, tile_inst.size() * sizeof(int))) &&
         (b->active = (uint8_t*)bdev_alloc(b, count)) &&
         (b->partial = (double*)bdev_alloc(b, (size_t)b->total_tiles * RED_NVAL * 8)) &&
         (b->red_out = (double*)bdev_alloc(b, (size_t)count * RED_NVAL * 8)) &&
         (b->barrier = (GridBarrier*)bdev_alloc(b, sizeof(GridBarrier))) &&
         (b->persist_err = (int*)bdev_alloc(b, sizeof(int)));
    if (ok && b->n_general)
        ok = (b->general = (int2*)bdev_alloc(b, general.size() * sizeof(int2))) &&
             (b->gen_nodes = (int*)bdev_alloc(b, gen_nodes.size() * sizeof(int))) &&
             (b->gen_tile_start = (int*)bdev_alloc(b, gen_start.size() * sizeof(int)));
    if (ok && b->n_dir)
        ok = (b->dirs = (DirNode*)bdev_alloc(b, dirs.size() * sizeof(DirNode))) &&
             (b->dir_owner = (int*)bdev_alloc(b, dir_owner.size() * sizeof(int)));
    if (ok && b->dir_fused) ok = (b->dir_start = (int*)bdev_alloc(b, dir_start.size() * sizeof(int))) != nullptr;
    if (!ok) {
        brelease(b);
        delete b;
        return bfail(nullptr, MACLAB_E_NOMEM, "device allocation failed");
    }
    // static data
    std::vector<double> D64(NP, 0.0);
    std::vector<uint8_t> type(NP + 64, 0);
    for (int i = 0; i < count; ++i) {
        std::copy(P[i].D64.begin(), P[i].D64.end(), D64.begin() + b->off[i]);
        std::copy(P[i].type.begin(), P[i].type.end(), type.begin() + b->off[i]);
    }
    cudaError_t ce = cudaSuccess;
    auto put = [&](void* dst, const void* src, size_t bytes) {
        if (ce == cudaSuccess && bytes) ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, b->stream);
    };
    put(b->D64, D64.data(), NP * 8);
    std::vector<float> Df;
    if (b->prec == MACLAB_F32) {
        Df.resize(NP);
        for (size_t k = 0; k < NP; ++k) Df[k] = (float)D64[k];
        put(b->D, Df.data(), NP * 4);
    } else {
        put(b->D, D64.data(), NP * 8);
    }
    put(b->type, type.data(), NP + 64);
    put(b->tile_inst, tile_inst.data(), tile_inst.size() * sizeof(int));
    if (b->n_general) {
        put(b->general, general.data(), general.size() * sizeof(int2));
        put(b->gen_nodes, gen_nodes.data(), gen_nodes.size() * sizeof(int));
        put(b->gen_tile_start, gen_start.data(), gen_start.size() * sizeof(int));
    }
    if (b->n_dir) {
        put(b->dirs, dirs.data(), dirs.size() * sizeof(DirNode));
        put(b->dir_owner, dir_owner.data(), dir_owner.size() * sizeof(int));
    }
    if (b->dir_fused) put(b->dir_start, dir_start.data(), dir_start.size() * sizeof(int));
    b->active_host.assign(count, 1);
    put(b->active, b->active_host.data(), count);
    std::vector<BatchInst<float>> instf;
    std::vector<BatchInst<double>> instd;
    if (b->prec == MACLAB_F32) {
        fill_insts<float>(b, P, instf);
        put(b->insts, instf.data(), instf.size() * sizeof(BatchInst<float>));
    } else {
        fill_insts<double>(b, P, instd);
        put(b->insts, instd.data(), instd.size() * sizeof(BatchInst<double>));
    }
    for (int k = 0; k < 2 && ce == cudaSuccess; ++k) {
        ce = cudaMemsetAsync(b->eta[k], 0, NP * b->esize, b->stream);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(b->u[k], 0, NP * b->esize, b->stream);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(b->v[k], 0, NP * b->esize, b->stream);
    }
    if (ce == cudaSuccess) ce = cudaMemsetAsync(b->persist_err, 0, sizeof(int), b->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(b->stream);
    if (ce == cudaSuccess)
        ce = b->prec == MACLAB_F32
            ? cudaFuncSetAttribute(step_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)tile::smem_bytes<float>())
            : cudaFuncSetAttribute(step_batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)tile::smem_bytes<double>());
    if (ce == cudaSuccess) ce = b->prec == MACLAB_F32 ? persistent_setup<float>(b) : persistent_setup<double>(b);
    if (ce != cudaSuccess) {
        bfail(nullptr, MACLAB_E_CUDA, std::string("batch upload: ") + cudaGetErrorString(ce));
        brelease(b);
        delete b;
        return MACLAB_E_CUDA;
    }
    *out = b;
    for (int i = 0; i < count; ++i) {
        if (h0 && h0[i]) {
            int rc = maclab_batch_set_state(b, i, h0[i], u0[i], v0[i]);
            if (rc != MACLAB_OK) {
                *out = nullptr;
                brelease(b);
                delete b;
                return rc;
            }
        }
    }
    b->have_prev = false;
    return MACLAB_OK;
}

int maclab_batch_step(maclab_batch_t b, int64_t n)
{
    if (!b) return bfail(nullptr, MACLAB_E_ARG, "NULL batch");
    if (int rc = batch_usable(b)) return rc;
    if (n < 0) return bfail(b, MACLAB_E_ARG, "n must be >= 0");
    if (use_persistent(b)) return b->prec == MACLAB_F32 ? batch_persistent<float>(b, n) : batch_persistent<double>(b, n);
    while (b->graph_steps > 0 && n >= b->graph_steps) {
        if (!b->graph[b->cur]) {
            int rc = batch_capture(b);
            if (rc != MACLAB_OK) return rc;
        }
        cudaError_t e = cudaGraphLaunch(b->graph[b->cur], b->stream);
        if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
        b->n += b->graph_steps;
        b->have_prev = true;
        n -= b->graph_steps;
    }
    for (int64_t k = 0; k < n; ++k) {
        int rc = batch_one(b, b->stream);
        if (rc != MACLAB_OK) return rc;
    }
    return MACLAB_OK;
}

int maclab_batch_set_graph_steps(maclab_batch_t b, int steps)
{
    if (!b) return bfail(nullptr, MACLAB_E_ARG, "NULL batch");
    if (steps < 0 || (steps & 1)) return bfail(b, MACLAB_E_ARG, "steps must be an even number >= 0");
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
        b->graph[k] = nullptr;
    }
    b->graph_steps = steps;
    return MACLAB_OK;
}

int maclab_batch_set_persistent(maclab_batch_t b, int mode)
{
    if (!b) return bfail(nullptr, MACLAB_E_ARG, "NULL batch");
    if (mode < 0 || mode > 1) return bfail(b, MACLAB_E_ARG, "mode must be 0 (one launch per step) or 1 (persistent)");
    b->persist_mode = mode;
    return MACLAB_OK;
}

int maclab_batch_residual(maclab_batch_t b, double* out)
{
    if (!b || !out) return bfail(b, MACLAB_E_ARG, "NULL argument");
    if (!b->have_prev) return bfail(b, MACLAB_E_STATE, "no step taken since create / set_state");
    const int prc = check_persist_err(b);
    if (prc != MACLAB_OK) return prc;
    if (int rc = batch_usable(b)) return rc;
    return b->prec == MACLAB_F32 ? batch_residual_t<float>(b, out) : batch_residual_t<double>(b, out);
}

int maclab_batch_mark(maclab_batch_t b)
{
    if (!b) return bfail(nullptr, MACLAB_E_ARG, "NULL batch");
    if (int rc = batch_usable(b)) return rc;
    const size_t bytes = b->total_np * b->esize;
    for (int k = 0; k < 3; ++k)
        if (!b->snap[k] && !(b->snap[k] = bdev_alloc(b, bytes))) return bfail(b, MACLAB_E_NOMEM, "mark: device memory");
    const void* src[3] = {b->eta[b->cur], b->u[b->cur], b->v[b->cur]};
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = cudaMemcpyAsync(b->snap[k], src[k], bytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("mark: ") + cudaGetErrorString(e));
    }
    b->mark_n = b->n;
    return MACLAB_OK;
}

int maclab_batch_residual_since_mark(maclab_batch_t b, double* out)
{
    if (!b || !out) return bfail(b, MACLAB_E_ARG, "NULL argument");
    if (b->mark_n < 0 || b->n <= b->mark_n) return bfail(b, MACLAB_E_STATE, "no marked state, or no step since it");
    const int prc = check_persist_err(b);
    if (prc != MACLAB_OK) return prc;
    if (int rc = batch_usable(b)) return rc;
    return b->prec == MACLAB_F32 ? batch_residual_t<float>(b, out, true) : batch_residual_t<double>(b, out, true);
}

int maclab_batch_set_active(maclab_batch_t b, const uint8_t* flags)
{
    if (!b || !flags) return bfail(b, MACLAB_E_ARG, "NULL argument");
    for (int i = 0; i < b->count; ++i) {
        const uint8_t f = flags[i] ? 1 : 0;
        if (!f && b->active_host[i]) {
            int rc = batch_freeze(b, i);
            if (rc != MACLAB_OK) return rc;
        }
        b->active_host[i] = f;
    }
    cudaError_t e = cudaMemcpyAsync(b->active, b->active_host.data(), b->count, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, MACLAB_E_CUDA, "batch set_active");
    return MACLAB_OK;
}

int maclab_batch_run_to_steady(maclab_batch_t b, double tol, int64_t max_steps, int check_every,
                               int64_t* steps, double* r_final, double* seconds)
{
    if (!b) return bfail(nullptr, MACLAB_E_ARG, "NULL batch");
    if (check_every < 1 || max_steps < 0 || !(tol >= 0)) return bfail(b, MACLAB_E_ARG, "bad tol / max_steps / check_every");
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<double> r(4 * (size_t)b->count, INFINITY);
    std::vector<uint8_t> act(b->active_host);
    std::vector<int64_t> done(b->count, -1);
    int64_t total = 0;
    int rc = MACLAB_OK;
    int remaining = 0;
    for (uint8_t a : act) remaining += a ? 1 : 0;
    while (remaining > 0 && total < max_steps) {
        const int64_t k = std::min<int64_t>(check_every, max_steps - total);
        if ((rc = maclab_batch_mark(b)) != MACLAB_OK) break;
        if ((rc = maclab_batch_step(b, k)) != MACLAB_OK) break;
        total += k;
        rc = maclab_batch_residual_since_mark(b, r.data());
        if (rc != MACLAB_OK) break;
        const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        bool changed = false;
        for (int i = 0; i < b->count; ++i) {
            if (act[i] && r[4 * i] <= tol) {
                act[i] = 0;
                done[i] = total;
                if (seconds) seconds[i] = secs;
                changed = true;
                --remaining;
            }
        }
        if (changed && (rc = maclab_batch_set_active(b, act.data())) != MACLAB_OK) break;
    }
    for (int i = 0; i < b->count; ++i) {
        if (steps) steps[i] = done[i];
        if (r_final) r_final[i] = r[4 * i];
    }
    if (rc == MACLAB_OK && remaining > 0) return bfail(b, MACLAB_E_STATE, "max_steps reached before every instance converged");
    return rc;
}

int maclab_batch_get_state(maclab_batch_t b, int i, double* h, double* u, double* v)
{
    if (!b || i < 0 || i >= b->count) return bfail(b, MACLAB_E_ARG, "bad instance");
    const int prc = check_persist_err(b);
    if (prc != MACLAB_OK) return prc;
    if (int rc = batch_usable(b)) return rc;
    const size_t N = (size_t)b->nx[i] * b->ny[i];
    const int c = b->cur;
    const size_t o = b->off[i];
    cudaError_t e = cudaSuccess;
    if (b->prec == MACLAB_F32)
        state_out_kernel<float><<<grid_blocks(N, 256, 4096), 256, 0, b->stream>>>(
            (const float*)b->eta[c] + o, (const float*)b->u[c] + o, (const float*)b->v[c] + o, b->D64 + o, b->stage,
            b->stage + N, b->stage + 2 * N, b->nx[i], b->ny[i], b->pitch[i]);
    else
        state_out_kernel<double><<<grid_blocks(N, 256, 4096), 256, 0, b->stream>>>(
            (const double*)b->eta[c] + o, (const double*)b->u[c] + o, (const double*)b->v[c] + o, b->D64 + o,
            b->stage, b->stage + N, b->stage + 2 * N, b->nx[i], b->ny[i], b->pitch[i]);
    if ((e = cudaGetLastError()) != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("batch get_state: ") + cudaGetErrorString(e));
    double* dst[3] = {h, u, v};
    for (int k = 0; k < 3; ++k)
        if (dst[k] && (e = cudaMemcpyAsync(dst[k], b->stage + k * N, N * 8, cudaMemcpyDeviceToHost, b->stream)) !=
                          cudaSuccess)
            return bfail(b, MACLAB_E_CUDA, std::string("batch get_state: ") + cudaGetErrorString(e));
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("batch get_state: ") + cudaGetErrorString(e));
    return MACLAB_OK;
}

int maclab_batch_device_state(maclab_batch_t b, int i, void** eta, void** u, void** v, int* pitch)
{
    if (!b || i < 0 || i >= b->count) return bfail(b, MACLAB_E_ARG, "bad instance");
    const int c = b->cur;
    const size_t o = b->off[i] * b->esize;
    if (eta) *eta = (char*)b->eta[c] + o;
    if (u) *u = (char*)b->u[c] + o;
    if (v) *v = (char*)b->v[c] + o;
    if (pitch) *pitch = b->pitch[i];
    return MACLAB_OK;
}

int maclab_batch_set_state(maclab_batch_t b, int i, const double* h, const double* u, const double* v)
{
    if (!b || i < 0 || i >= b->count || !h || !u || !v) return bfail(b, MACLAB_E_ARG, "bad instance or NULL state");
    const size_t N = (size_t)b->nx[i] * b->ny[i];
    const size_t o = b->off[i];
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->stage, h, N * 8, cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->stage + N, u, N * 8, cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->stage + 2 * N, v, N * 8, cudaMemcpyHostToDevice, b->stream)) != cudaSuccess)
        return bfail(b, MACLAB_E_CUDA, std::string("batch set_state: ") + cudaGetErrorString(e));
    const int c = b->cur, d = 1 - b->cur;
    // both buffers: the instance is consistent whatever the parity
    if (b->prec == MACLAB_F32)
        state_in_kernel<float><<<grid_blocks(N, 256, 4096), 256, 0, b->stream>>>(
            b->stage, b->stage + N, b->stage + 2 * N, b->D64 + o, b->type + o, (float*)b->eta[c] + o,
            (float*)b->u[c] + o, (float*)b->v[c] + o, (float*)b->eta[d] + o, (float*)b->u[d] + o,
            (float*)b->v[d] + o, b->nx[i], b->ny[i], b->pitch[i]);
    else
        state_in_kernel<double><<<grid_blocks(N, 256, 4096), 256, 0, b->stream>>>(
            b->stage, b->stage + N, b->stage + 2 * N, b->D64 + o, b->type + o, (double*)b->eta[c] + o,
            (double*)b->u[c] + o, (double*)b->v[c] + o, (double*)b->eta[d] + o, (double*)b->u[d] + o,
            (double*)b->v[d] + o, b->nx[i], b->ny[i], b->pitch[i]);
    if ((e = cudaGetLastError()) != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("batch set_state: ") + cudaGetErrorString(e));
    if ((e = cudaStreamSynchronize(b->stream)) != cudaSuccess) return bfail(b, MACLAB_E_CUDA, std::string("batch set_state: ") + cudaGetErrorString(e));
    int rc = batch_freeze(b, i);
    if (rc == MACLAB_OK && (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
        return bfail(b, MACLAB_E_CUDA, std::string("batch set_state: ") + cudaGetErrorString(e));
    b->have_prev = false;
    b->mark_n = -1;  // the mark belongs to the replaced history
    if (rc == MACLAB_OK && b->broken) {
        // usable again once every instance holds a state set by the caller
        b->reloaded[i] = 1;
        bool all = true;
        for (uint8_t r : b->reloaded) all = all && r;
        if (all) {
            if ((e = cudaMemsetAsync(b->persist_err, 0, sizeof(int), b->stream)) != cudaSuccess ||
                (e = cudaStreamSynchronize(b->stream)) != cudaSuccess)
                return bfail(b, MACLAB_E_CUDA, std::string("batch set_state: ") + cudaGetErrorString(e));
            b->broken = false;
        }
    }
    return rc;
}

int maclab_batch_set_barrier_test(maclab_batch_t b, int extra, unsigned int polls)
{
    if (!b) return bfail(nullptr, MACLAB_E_ARG, "NULL batch");
    if (extra < 0 || polls < 1) return bfail(b, MACLAB_E_ARG, "extra must be >= 0 and polls >= 1");
    b->bar_extra = (unsigned int)extra;
    b->bar_polls = polls;
    return MACLAB_OK;
}

int maclab_batch_info(maclab_batch_t b, int* count, int64_t* nodes, int64_t* tiles, int64_t* steps)
{
    if (!b) return bfail(nullptr, MACLAB_E_ARG, "NULL batch");
    int64_t tot = 0;
    for (int64_t x : b->nodes) tot += x;
    if (count) *count = b->count;
    if (nodes) *nodes = tot;
    if (tiles) *tiles = b->total_tiles;
    if (steps) *steps = b->n;
    return MACLAB_OK;
}

const char* maclab_batch_last_error(maclab_batch_t b) { return b ? b->err.c_str() : g_last_error.c_str(); }

void maclab_batch_destroy(maclab_batch_t b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    brelease(b);
    delete b;
}

}  // extern "C"
