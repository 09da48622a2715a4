// warmstart.cu -- learned warm start (include/maclab_ws.h): a residual
// convolutional network on a coarse grid, trained on steady states of the
// plain iteration, proposing the starting state of a steady-state run.
//
// Every convolution is an implicit GEMM on the tensor cores with bfloat16
// operands and float accumulators:
//   by default (tensor_path = 0) every convolution (forward and input
//     gradient, the 16-channel input and output layers included) and every
//     weight gradient runs on tcgen05.mma with operands brought in by TMA
//     tensor copies into swizzled shared memory, accumulators in tensor
//     memory, copies, MMAs and the epilogue in warps of their own
//     (ws_conv5_kernel, ws_wgrad5_kernel in ws_tc5.cuh);
//   tensor_path = 1 runs the 128 -> 128 convolutions on tcgen05 with
//     operands staged by cp.async in the canonical no-swizzle K-major layout
//     (ws_conv_tc_kernel, slower: its per-thread copies set its pace), the
//     rest on mma.sync;
//   tensor_path = 2 runs everything on mma.sync m16n8k16 with ldmatrix
//     fragment loads (ws_conv_kernel, ws_wgrad_kernel);
//   forward / input gradient: M = pixels, N = output channels,
//     K = 9 taps x input channels;
//   weight gradient: M and N the two channel sides, K = pixels (split over
//     blocks, the splits' sums added in order afterwards).
#include "maclab.h"
#include "maclab_ws.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

void maclab_note_error(const std::string& msg);

namespace {

using bf16 = __nv_bfloat16;
constexpr int IO = MACLAB_WS_IO;
constexpr int CELL = MACLAB_WS_CELL;
constexpr int THREADS = 256;

// ---------------------------------------------------------------------------
// PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, bool valid)
{
    const int n = valid ? 16 : 0;  // 0: the 16 bytes are filled with zeros
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], uint32_t a)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm2(uint32_t (&r)[2], uint32_t a)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], uint32_t a)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm2t(uint32_t (&r)[2], uint32_t a)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
// D += A B, A 16 x 16 (row), B 16 x 8 (col), bfloat16 in, float accumulate
__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t relu2(uint32_t x)
{
    __nv_bfloat162 v;
    memcpy(&v, &x, 4);
    v = __hmax2(v, __float2bfloat162_rn(0.f));
    uint32_t r;
    memcpy(&r, &v, 4);
    return r;
}

// ---------------------------------------------------------------------------
// Convolution as implicit GEMM (forward, and input gradient with flipped,
// transposed weights).  A block computes 64 pixels of one image row
// (x0 .. x0 + 63 of row y of image b) times NT output channels.
//   X  [B][R][R][Cin] bf16;  Wk [9][Cout][Cin] bf16 (the B operand, K
//   contiguous per output channel)
//   epilogue: v = acc + bias; v = gate > 0 ? v : 0 (gate [B][R][R][Cout]);
//   v += res; Y (bf16) and / or Yf (float) [B][R][R][Cout]
struct ConvArgs {
    const bf16* X;
    const bf16* Wk;
    const float* bias;
    const bf16* gate;
    const bf16* res;
    bf16* Y;
    float* Yf;
    int R, Cin, Cout, dil, relu_in;
};

constexpr int CONV_M = 64;
constexpr int CONV_STAGES = 3;

// 16-byte chunk h (0, 1) of 32-byte row r, swizzled so that ldmatrix rows
// r .. r + 7 fall in distinct bank groups
__device__ __forceinline__ int swz32(int r, int h) { return r * 32 + ((h ^ ((r >> 2) & 1)) << 4); }

template <int NT>
__global__ void __launch_bounds__(THREADS) ws_conv_kernel(const ConvArgs a)
{
    constexpr int WN = NT / 2;           // output channels per warp (2 warps along N)
    constexpr int NJ = WN / 8;           // n8 tiles per warp
    __shared__ __align__(128) unsigned char sA[CONV_STAGES][CONV_M * 32];
    __shared__ __align__(128) unsigned char sB[CONV_STAGES][NT * 32];
    const int R = a.R, Cin = a.Cin, Cout = a.Cout, dil = a.dil;
    const int segs = R / CONV_M;
    const int row = blockIdx.x / segs;   // b * R + y
    const int x0 = (blockIdx.x % segs) * CONV_M;
    const int b = row / R, y = row % R;
    const int n0 = blockIdx.y * NT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int kci = Cin / 16;
    const int KT = 9 * kci;

    auto load = [&](int stage, int kk) {
        const int tap = kk / kci, ci0 = (kk % kci) * 16;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        if (tid < CONV_M * 2) {
            const int m = tid >> 1, h = tid & 1;
            const int yy = y + dy * dil, xx = x0 + m + dx * dil;
            const bool ok = yy >= 0 && yy < R && xx >= 0 && xx < R;
            const bf16* src = ok ? a.X + ((size_t)(b * R + yy) * R + xx) * Cin + ci0 + h * 8 : a.X;
            cp16(smem_addr(&sA[stage][swz32(m, h)]), src, ok);
        }
        for (int i = tid; i < NT * 2; i += THREADS) {
            const int n = i >> 1, h = i & 1;
            const bf16* src = a.Wk + ((size_t)tap * Cout + n0 + n) * Cin + ci0 + h * 8;
            cp16(smem_addr(&sB[stage][swz32(n, h)]), src, true);
        }
    };

    float acc[NJ][4];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

#pragma unroll
    for (int s = 0; s < CONV_STAGES - 1; ++s) {
        if (s < KT) load(s, s);
        cp_commit();
    }
    for (int kk = 0; kk < KT; ++kk) {
        cp_wait<CONV_STAGES - 2>();
        __syncthreads();
        const int pf = kk + CONV_STAGES - 1;
        if (pf < KT) load(pf % CONV_STAGES, pf);
        cp_commit();
        const int st = kk % CONV_STAGES;
        uint32_t af[4];
        {
            const int r = wm * 16 + (lane & 15), h = lane >> 4;
            ldsm4(af, smem_addr(&sA[st][swz32(r, h)]));
        }
        if (a.relu_in) {
#pragma unroll
            for (int q = 0; q < 4; ++q) af[q] = relu2(af[q]);
        }
        if constexpr (NJ >= 2) {
#pragma unroll
            for (int j = 0; j < NJ; j += 2) {
                const int n = wn * WN + j * 8 + (lane & 7) + ((lane >> 4) << 3), h = (lane >> 3) & 1;
                uint32_t bq[4];
                ldsm4(bq, smem_addr(&sB[st][swz32(n, h)]));
                const uint32_t b0[2] = {bq[0], bq[1]}, b1[2] = {bq[2], bq[3]};
                mma(acc[j], af, b0);
                mma(acc[j + 1], af, b1);
            }
        } else {
            const int n = wn * WN + (lane & 7), h = (lane >> 3) & 1;
            uint32_t bq[2];
            ldsm2(bq, smem_addr(&sB[st][swz32(n, h)]));
            mma(acc[0], af, bq);
        }
    }
    cp_wait<0>();

    // epilogue: fragment (row g / g + 8, columns 2c, 2c + 1) of each n8 tile
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int n = n0 + wn * WN + j * 8 + 2 * c;
        const float b0 = a.bias ? a.bias[n] : 0.f, b1 = a.bias ? a.bias[n + 1] : 0.f;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int m = wm * 16 + g + 8 * hh;
            const size_t o = ((size_t)row * R + x0 + m) * Cout + n;
            float v0 = acc[j][2 * hh] + b0, v1 = acc[j][2 * hh + 1] + b1;
            if (a.gate) {
                const __nv_bfloat162 gt = *reinterpret_cast<const __nv_bfloat162*>(a.gate + o);
                if (!(__bfloat162float(gt.x) > 0.f)) v0 = 0.f;
                if (!(__bfloat162float(gt.y) > 0.f)) v1 = 0.f;
            }
            if (a.res) {
                const __nv_bfloat162 rr = *reinterpret_cast<const __nv_bfloat162*>(a.res + o);
                v0 += __bfloat162float(rr.x);
                v1 += __bfloat162float(rr.y);
            }
            if (a.Y) *reinterpret_cast<__nv_bfloat162*>(a.Y + o) = __floats2bfloat162_rn(v0, v1);
            if (a.Yf) *reinterpret_cast<float2*>(a.Yf + o) = make_float2(v0, v1);
        }
    }
}

// ---------------------------------------------------------------------------
// The same convolution on tcgen05: a block owns 128 consecutive pixels of
// one image (M = 128) and 128 output channels (N = 128); K runs over the 9
// taps x input channels in stages of TC_KS channels of one tap (TC_KS / 16
// MMAs of K = 16).  TC_STAGES operand buffers rotate: the copies of a stage
// are issued TC_STAGES - 1 stages ahead (the MMAs of a stage take far less
// time than its copies), one thread issues each stage's MMAs, and
// tcgen05.commit signals the stage's mbarrier when its MMAs are done with
// the buffer.
//   shared-memory operand layout (K-major, no swizzle): 8 x 8 core matrices
//   of 128 bytes (8 rows of 16 bytes); core matrix (row group g, K chunk kc)
//   at kc * 2048 + g * 128, so the descriptor's leading (K) byte offset is
//   2048 and its stride (8-row group) byte offset 128.
#ifndef MACLAB_TC_KS
#define MACLAB_TC_KS 32
#endif
#ifndef MACLAB_TC_STAGES
#define MACLAB_TC_STAGES 6
#endif
constexpr int TC_M = 128, TC_N = 128, TC_KS = MACLAB_TC_KS, TC_THREADS = 256, TC_STAGES = MACLAB_TC_STAGES;
constexpr uint32_t TC_OPER = TC_M * TC_KS * 2;          // bytes per operand and stage
constexpr size_t TC_SMEM = TC_STAGES * 2 * TC_OPER + 1024;  // stages x (A, B) + alignment slack
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;
// instruction descriptor, kind::f16: f32 accumulate, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint32_t tc_off(int row, int kc) { return kc * 2048 + (row >> 3) * 128 + (row & 7) * 16; }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(2048 >> 4) << 16;  // leading byte offset: next core matrix along K
    d |= (uint64_t)(128 >> 4) << 32;   // stride byte offset: next group of 8 rows
    d |= (uint64_t)1 << 46;            // descriptor version of this tensor-core generation
    return d;                          // base offset 0, no swizzle
}

__device__ __forceinline__ void tc_mbar_init(uint32_t bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool tc_mbar_wait(uint32_t bar, uint32_t phase)
{
    for (uint32_t k = 0; k < TC_WAIT_LIMIT; ++k) {
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

__global__ void __launch_bounds__(TC_THREADS) ws_conv_tc_kernel(const ConvArgs a, int* err)
{
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    __shared__ __align__(8) uint64_t mbar[TC_STAGES];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    // operand buffers on a 1024-byte boundary
    const uint32_t raw = smem_addr(tsm_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* tsm = tsm_raw + (base - raw);
    const int R = a.R, Cin = a.Cin, Cout = a.Cout, dil = a.dil;
    const int P = R * R, tiles = P / TC_M;
    const int b = blockIdx.x / tiles, p0 = (blockIdx.x % tiles) * TC_M;
    const int n0 = blockIdx.y * TC_N;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_slot)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < TC_STAGES; ++k) tc_mbar_init(smem_addr(&mbar[k]));
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int kch = Cin / TC_KS;
    const int KT = 9 * kch;
    uint32_t phase[TC_STAGES];
#pragma unroll
    for (int k = 0; k < TC_STAGES; ++k) phase[k] = 0;

    auto load = [&](int kk) {
        const int buf = kk % TC_STAGES;
        const int tap = kk / kch, ci0 = (kk % kch) * TC_KS;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        unsigned char* A = tsm + buf * 2 * TC_OPER;
        unsigned char* Bm = A + TC_OPER;
        for (int i = tid; i < TC_M * (TC_KS / 8); i += TC_THREADS) {
            const int m = i / (TC_KS / 8), kc = i % (TC_KS / 8);
            const int p = p0 + m, y = p / R, x = p % R;
            const int yy = y + dy * dil, xx = x + dx * dil;
            const bool in = yy >= 0 && yy < R && xx >= 0 && xx < R;
            const bf16* src = in ? a.X + ((size_t)(b * R + yy) * R + xx) * Cin + ci0 + kc * 8 : a.X;
            cp16(smem_addr(A + tc_off(m, kc)), src, in);
            const bf16* wsrc = a.Wk + ((size_t)tap * Cout + n0 + m) * Cin + ci0 + kc * 8;
            cp16(smem_addr(Bm + tc_off(m, kc)), wsrc, true);
        }
    };

    bool ok = true;
#pragma unroll
    for (int s = 0; s < TC_STAGES - 1; ++s) {
        if (s < KT) load(s);
        cp_commit();
    }
    for (int kk = 0; kk < KT; ++kk) {
        const int pf = kk + TC_STAGES - 1;
        if (pf < KT) {
            // buffer pf % TC_STAGES was last read by the MMAs of stage kk - 1
            if (kk >= 1) {
                const int pb = (kk - 1) % TC_STAGES;
                if (!tc_mbar_wait(smem_addr(&mbar[pb]), phase[pb])) atomicOr(&abort_flag, 1);
                phase[pb] ^= 1u;
                __syncthreads();
                if (abort_flag) {
                    ok = false;
                    break;
                }
            }
            load(pf);
        }
        cp_commit();
        cp_wait<TC_STAGES - 1>();  // this thread's copies of stage kk have landed
        const int buf = kk % TC_STAGES;
        unsigned char* A = tsm + buf * 2 * TC_OPER;
        if (a.relu_in) {  // each thread rectifies the chunks it staged
            for (int i = tid; i < TC_M * (TC_KS / 8); i += TC_THREADS) {
                uint4* q = reinterpret_cast<uint4*>(A + tc_off(i / (TC_KS / 8), i % (TC_KS / 8)));
                uint4 v = *q;
                v.x = relu2(v.x);
                v.y = relu2(v.y);
                v.z = relu2(v.z);
                v.w = relu2(v.w);
                *q = v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // staged data visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t sa = smem_addr(A), sb = sa + TC_OPER;
#pragma unroll
            for (int k16 = 0; k16 < TC_KS / 16; ++k16) {
                const uint64_t ad = tc_desc(sa + k16 * 2 * 2048), bd = tc_desc(sb + k16 * 2 * 2048);
                const uint32_t acc = (kk > 0 || k16 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_addr(&mbar[buf]))
                         : "memory");
        }
    }
    cp_wait<0>();
    // the last commit covers every MMA issued before it
    if (ok && KT > 0) {
        const int lb = (KT - 1) % TC_STAGES;
        if (!tc_mbar_wait(smem_addr(&mbar[lb]), phase[lb])) atomicOr(&abort_flag, 1);
        __syncthreads();
        ok = !abort_flag;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31
        // (pixels), columns 64 (w / 4) .. + 63
        const int m = (warp & 3) * 32 + lane;
        const int cbase = (warp >> 2) * (TC_N / 2);
        const size_t orow = ((size_t)b * P + p0 + m) * Cout + n0;
#pragma unroll 1
        for (int c0 = cbase; c0 < cbase + TC_N / 2; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                const int n = n0 + c0 + j;
                const size_t o = orow + c0 + j;
                float v0 = __uint_as_float(r[j]) + (a.bias ? a.bias[n] : 0.f);
                float v1 = __uint_as_float(r[j + 1]) + (a.bias ? a.bias[n + 1] : 0.f);
                if (a.gate) {
                    const __nv_bfloat162 gt = *reinterpret_cast<const __nv_bfloat162*>(a.gate + o);
                    if (!(__bfloat162float(gt.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(gt.y) > 0.f)) v1 = 0.f;
                }
                if (a.res) {
                    const __nv_bfloat162 rr = *reinterpret_cast<const __nv_bfloat162*>(a.res + o);
                    v0 += __bfloat162float(rr.x);
                    v1 += __bfloat162float(rr.y);
                }
                if (a.Y) *reinterpret_cast<__nv_bfloat162*>(a.Y + o) = __floats2bfloat162_rn(v0, v1);
                if (a.Yf) *reinterpret_cast<float2*>(a.Yf + o) = make_float2(v0, v1);
            }
        }
    } else if (tid == 0) {
        // a wait gave up: let the MMAs already issued finish (bounded) before
        // the accumulator is released
        atomicOr(err, 1);
        for (int k = 0; k < TC_STAGES; ++k) tc_mbar_wait(smem_addr(&mbar[k]), phase[k]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_N) : "memory");
}

// ---------------------------------------------------------------------------
// Tensor maps of the TMA-fed tcgen05 kernels (ws_tc5.cuh): A and B operand
// of a convolution, or output gradient and input of a weight gradient.
struct TmaOperands {
    CUtensorMap A;
    CUtensorMap B;
};

// ---------------------------------------------------------------------------
// Weight gradient: dW[tap][co][ci] += sum_p dY[p][co] * act(X)[p + off(tap)][ci]
// A block owns one tap, an MT x NT tile of (co, ci) and every split-th
// chunk of 32 pixels.
struct WgradArgs {
    const bf16* dY;   // [B][R][R][Cout]
    const bf16* X;    // [B][R][R][Cin]
    float* dW;        // [9][Cout][Cin]
    float* part;      // [splits][9][Cout][Cin]: each split's sums, added in order afterwards
    int B, R, Cin, Cout, dil, relu_in, splits;
};
constexpr int WG_K = 32;  // pixels per stage

// 16-byte chunk h of row r when a row holds `chunks` chunks (2 or 8)
__device__ __forceinline__ int swz_rows(int r, int h, int chunks)
{
    return chunks == 8 ? r * 128 + ((h ^ (r & 7)) << 4) : r * 32 + ((h ^ ((r >> 2) & 1)) << 4);
}

template <int MT, int NT>
__global__ void __launch_bounds__(THREADS) ws_wgrad_kernel(const WgradArgs a)
{
    constexpr int WMW = MT / 16;         // warps along M
    constexpr int WNW = 8 / WMW;         // warps along N
    constexpr int WN = NT / WNW;         // ci per warp
    constexpr int NJ = WN / 8;
    constexpr int CA = MT / 8, CB = NT / 8;  // 16-byte chunks per staged row
    __shared__ __align__(128) unsigned char sA[2][WG_K * MT * 2];
    __shared__ __align__(128) unsigned char sB[2][WG_K * NT * 2];
    const int R = a.R, Cin = a.Cin, Cout = a.Cout, dil = a.dil;
    const int mt = Cout / MT;
    const int tile = blockIdx.x;
    const int m0 = (tile % mt) * MT, k0 = (tile / mt) * NT;
    const int tap = blockIdx.y, split = blockIdx.z;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp % WMW, wn = warp / WMW;
    const int chunks_total = a.B * R * R / WG_K;

    auto load = [&](int stage, int ch) {
        const int p0 = ch * WG_K;            // first pixel (b, y, x0)
        const int rowi = p0 / R, x0 = p0 % R;
        const int b = rowi / R, y = rowi % R;
        for (int i = tid; i < WG_K * CA; i += THREADS) {
            const int r = i / CA, h = i % CA;
            const bf16* src = a.dY + (size_t)(p0 + r) * Cout + m0 + h * 8;
            cp16(smem_addr(&sA[stage][swz_rows(r, h, CA)]), src, true);
        }
        const int yy = y + dy * dil;
        for (int i = tid; i < WG_K * CB; i += THREADS) {
            const int r = i / CB, h = i % CB;
            const int xx = x0 + r + dx * dil;
            const bool ok = yy >= 0 && yy < R && xx >= 0 && xx < R;
            const bf16* src = ok ? a.X + ((size_t)(b * R + yy) * R + xx) * Cin + k0 + h * 8 : a.X;
            cp16(smem_addr(&sB[stage][swz_rows(r, h, CB)]), src, ok);
        }
    };

    float acc[NJ][4];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

    int ch = split;
    if (ch < chunks_total) load(0, ch);
    cp_commit();
    int st = 0;
    for (; ch < chunks_total; ch += a.splits) {
        const int nx = ch + a.splits;
        if (nx < chunks_total) load(st ^ 1, nx);
        cp_commit();
        cp_wait<1>();
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < WG_K / 16; ++ks) {
            uint32_t af[4];
            {
                // A = dY^T: rows co, columns pixels; staged [pixel][co]
                const int r = ks * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int h = (wm * 16 + ((lane >> 3) & 1) * 8) / 8;
                ldsm4t(af, smem_addr(&sA[st][swz_rows(r, h, CA)]));
            }
            if constexpr (NJ >= 2) {
#pragma unroll
                for (int j = 0; j < NJ; j += 2) {
                    const int r = ks * 16 + (lane & 7) + (((lane >> 3) & 1) << 3);
                    const int h = (wn * WN + j * 8 + ((lane >> 4) << 3)) / 8;
                    uint32_t bq[4];
                    ldsm4t(bq, smem_addr(&sB[st][swz_rows(r, h, CB)]));
                    if (a.relu_in) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) bq[q] = relu2(bq[q]);
                    }
                    const uint32_t b0[2] = {bq[0], bq[1]}, b1[2] = {bq[2], bq[3]};
                    mma(acc[j], af, b0);
                    mma(acc[j + 1], af, b1);
                }
            } else {
                const int r = ks * 16 + (lane & 7) + (((lane >> 3) & 1) << 3);
                const int h = (wn * WN) / 8;
                uint32_t bq[2];
                ldsm2t(bq, smem_addr(&sB[st][swz_rows(r, h, CB)]));
                if (a.relu_in) {
                    bq[0] = relu2(bq[0]);
                    bq[1] = relu2(bq[1]);
                }
                mma(acc[0], af, bq);
            }
        }
        __syncthreads();  // stage st is free before the next load into it
        st ^= 1;
    }
    cp_wait<0>();
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int n = k0 + wn * WN + j * 8 + 2 * c;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int m = m0 + wm * 16 + g + 8 * hh;
            float* d = a.part + (((size_t)split * 9 + tap) * Cout + m) * Cin + n;
            *reinterpret_cast<float2*>(d) = make_float2(acc[j][2 * hh], acc[j][2 * hh + 1]);
        }
    }
}

#include "ws_tc5.cuh"

// out[i] = sum over s < S of part[s n + i], added in the order of s, so that
// split sums combine the same way in every run; eight loads are issued
// before their additions
__global__ void ws_sum_parts_kernel(const float* __restrict__ part, int S, size_t n, float* __restrict__ out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float t = 0.f;
        int s = 0;
        for (; s + 8 <= S; s += 8) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = part[(size_t)(s + j) * n + i];
#pragma unroll
            for (int j = 0; j < 8; ++j) t += v[j];
        }
        for (; s < S; ++s) t += part[(size_t)s * n + i];
        out[i] = t;
    }
}

// out[c] = sum over b < nb of part[b k + c], c < k, in the order of b
// out[c] = sum over b < nb of part[b k + c], c < k: one block per c, the
// threads' strided sums then a tree in shared memory, the same order in
// every run
__global__ void __launch_bounds__(THREADS) ws_sum_doubles_kernel(const double* __restrict__ part, int nb, int k,
                                                                 double* __restrict__ out)
{
    __shared__ double red[THREADS];
    const int c = blockIdx.x;
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += THREADS) t += part[(size_t)b * k + c];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int h = THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// out_part[blockIdx.x][c] = sum of dY[p][c] over the block's share of the
// P pixels: thread (lane l, group g) adds 8 channels (one 16-byte vector)
// of every (THREADS / (C / 8))-th pixel, then the lanes' sums are added in
// lane order; C a multiple of 8, at most 8 THREADS
constexpr int BG_BLOCKS = 256;
__global__ void __launch_bounds__(THREADS) ws_bias_grad_kernel(const bf16* __restrict__ dY, int P, int C,
                                                               float* __restrict__ out_part)
{
    __shared__ float red[THREADS * 8];
    const int G = C / 8, L = THREADS / G;
    const int g = threadIdx.x % G, l = threadIdx.x / G;
    const int p0 = (int)((long long)blockIdx.x * P / gridDim.x), p1 = (int)((long long)(blockIdx.x + 1) * P / gridDim.x);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto add = [&](const uint4& q) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[2 * j] += __bfloat162float(h[j].x);
            acc[2 * j + 1] += __bfloat162float(h[j].y);
        }
    };
    if (l < L) {
        int p = p0 + l;
        for (; p + 3 * L < p1; p += 4 * L) {  // four loads in flight, added in pixel order
            uint4 q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) q[u] = *reinterpret_cast<const uint4*>(dY + (size_t)(p + u * L) * C + g * 8);
#pragma unroll
            for (int u = 0; u < 4; ++u) add(q[u]);
        }
        for (; p < p1; p += L) add(*reinterpret_cast<const uint4*>(dY + (size_t)p * C + g * 8));
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[threadIdx.x * 8 + j] = acc[j];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += THREADS) {
        float t = 0.f;
        for (int k = 0; k < L; ++k) t += red[k * G * 8 + c];
        out_part[(size_t)blockIdx.x * C + c] = t;
    }
}

// loss = sum_p w_p sum_{c < oc} (Y - T)^2: block partials in double into
// loss_part[blockIdx.x]; dY = 2 w (Y - T) for c < oc, 0 otherwise
__global__ void __launch_bounds__(THREADS) ws_loss_kernel(const float* Y, const float* T, const float* W, int P,
                                                          int oc, bf16* dY, double* loss_part)
{
    __shared__ double part[THREADS];
    double s = 0.0;
    for (int i = blockIdx.x * THREADS + threadIdx.x; i < P * IO; i += gridDim.x * THREADS) {
        const int p = i / IO, c = i % IO;
        float g = 0.f;
        if (c < oc) {
            const float d = Y[i] - T[i];
            s += (double)W[p] * d * d;
            g = 2.f * W[p] * d;
        }
        dY[i] = __float2bfloat16_rn(g);
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int k = THREADS / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) part[threadIdx.x] += part[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = part[0];
}

// bf16 -> float
__global__ void ws_from_bf16_kernel(const bf16* x, float* y, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __bfloat162float(x[i]);
}

// float -> bf16
__global__ void ws_to_bf16_kernel(const float* x, bf16* y, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// Adam on the flat parameter vector; lr_t carries the bias corrections
// Layers of the parameter vector for ws_update_kernel: where each layer's
// weights start, and its channel counts (at most 64 blocks + lift + head).
constexpr int WS_MAX_LAYERS = 66;
struct LayerTable {
    int n;
    long long w_off[WS_MAX_LAYERS];
    int cin[WS_MAX_LAYERS], cout[WS_MAX_LAYERS];
};

// One pass over the parameter vector: with adam, one Adam step (lr_t
// carries the bias corrections); then every weight is packed in bfloat16
// twice, Wf[tap][co][ci] for the forward convolution and Wb[8 - tap][ci][co]
// (taps mirrored, channels swapped) for the input gradient, both at the
// weight's own offset in the parameter vector (biases leave gaps).
__global__ void ws_update_kernel(float* p, const float* g, float* m, float* v, size_t n, int adam, float lr_t,
                                 float b1, float b2, float eps, const __grid_constant__ LayerTable tab, bf16* Wf,
                                 bf16* Wb)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float pi = p[i];
        if (adam) {
            const float gi = g[i];
            const float mi = b1 * m[i] + (1.f - b1) * gi;
            const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            pi -= lr_t * mi / (sqrtf(vi) + eps);
            p[i] = pi;
        }
        int lo = 0, hi = tab.n - 1;  // the last layer starting at or before i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tab.w_off[mid] <= (long long)i) lo = mid;
            else hi = mid - 1;
        }
        const long long k = (long long)i - tab.w_off[lo];
        const int Cin = tab.cin[lo], Cout = tab.cout[lo];
        if (k < 9LL * Cin * Cout) {
            const int ci = (int)(k % Cin), co = (int)((k / Cin) % Cout), t = (int)(k / ((long long)Cin * Cout));
            const bf16 w = __float2bfloat16_rn(pi);
            Wf[i] = w;
            Wb[tab.w_off[lo] + ((long long)(8 - t) * Cin + ci) * Cout + co] = w;
        }
    }
}


// ---------------------------------------------------------------------------
// Fine grid <-> coarse grid
__global__ void ws_encode_kernel(int n, int R, const float* D, const uint8_t* mask, float wu, float wv, float cb,
                                 float dx, const float* eta, const float* u, const float* v, int pitch, float s0, float s1,
                                 float s2, float s3, float* X, float* T, float* Wt)
{
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= R * R) return;
    const int I = cell % R, J = cell / R;
    float cnt = 0.f, sd = 0.f, se = 0.f, su = 0.f, sv = 0.f;
    for (int j = J * CELL; j < J * CELL + CELL; ++j)
        for (int i = I * CELL; i < I * CELL + CELL; ++i) {
            const size_t k = (size_t)j * n + i;
            if (mask[k] == MACLAB_SOLID) continue;
            cnt += 1.f;
            sd += D[k];
            if (eta) {
                const size_t q = (size_t)j * pitch + i;
                se += eta[q];
                su += u[q];
                sv += v[q];
            }
        }
    const float inv = cnt > 0.f ? 1.f / cnt : 0.f;
    float* x = X + (size_t)cell * IO;
    x[0] = cnt / (CELL * CELL);
    x[1] = sd * inv / s0;
    x[2] = wu / 5.f;
    x[3] = wv / 5.f;
    x[4] = 100.f * cb;
    x[5] = 2.f * (I + 0.5f) / R - 1.f;
    x[6] = 2.f * (J + 0.5f) / R - 1.f;
    x[7] = 0.5f * dx;
    for (int c = 8; c < IO; ++c) x[c] = 0.f;
    if (T) {
        float* t = T + (size_t)cell * IO;
        t[0] = se * inv / s1;
        t[1] = su * inv / s2;
        t[2] = sv * inv / s3;
        for (int c = 3; c < IO; ++c) t[c] = 0.f;
        Wt[cell] = cnt / (CELL * CELL);
    }
}

__global__ void ws_decode_kernel(int n, int R, const float* Y, const float* D, const uint8_t* mask, double s1,
                                 double s2, double s3, double* h, double* u, double* v)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * n) return;
    const int i = k % n, j = k / n;
    const uint8_t t = mask[k];
    if (t == MACLAB_SOLID) {
        h[k] = D[k];
        u[k] = 0.0;
        v[k] = 0.0;
        return;
    }
    // coarse coordinates of the node (cell centres at integers), clamped
    const float fx = fminf(fmaxf((i + 0.5f) / CELL - 0.5f, 0.f), R - 1.f);
    const float fy = fminf(fmaxf((j + 0.5f) / CELL - 0.5f, 0.f), R - 1.f);
    const int x0 = min((int)fx, R - 2), y0 = min((int)fy, R - 2);
    const int x1 = x0 + 1, y1 = y0 + 1;
    const float ax = fx - x0, ay = fy - y0;
    float out[3];
    for (int c = 0; c < 3; ++c) {
        const float a00 = Y[((size_t)y0 * R + x0) * IO + c], a10 = Y[((size_t)y0 * R + x1) * IO + c];
        const float a01 = Y[((size_t)y1 * R + x0) * IO + c], a11 = Y[((size_t)y1 * R + x1) * IO + c];
        out[c] = (1.f - ay) * ((1.f - ax) * a00 + ax * a10) + ay * ((1.f - ax) * a01 + ax * a11);
    }
    h[k] = (double)D[k] + out[0] * s1;
    const bool still = t == MACLAB_NOSLIP;
    u[k] = still ? 0.0 : out[1] * s2;
    v[k] = still ? 0.0 : out[2] * s3;
}

// sum over non-solid nodes of (h - D) and their count: block partials into
// part[2 blockIdx.x], part[2 blockIdx.x + 1]
__global__ void __launch_bounds__(THREADS) ws_eta_sum_kernel(int nn, const double* h, const float* D,
                                                             const uint8_t* mask, double* part)
{
    __shared__ double ps[THREADS], pc[THREADS];
    double s = 0.0, c = 0.0;
    for (int k = blockIdx.x * THREADS + threadIdx.x; k < nn; k += gridDim.x * THREADS)
        if (mask[k] != MACLAB_SOLID) {
            s += h[k] - (double)D[k];
            c += 1.0;
        }
    ps[threadIdx.x] = s;
    pc[threadIdx.x] = c;
    __syncthreads();
    for (int k = THREADS / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            ps[threadIdx.x] += ps[threadIdx.x + k];
            pc[threadIdx.x] += pc[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ps[0];
        part[2 * blockIdx.x + 1] = pc[0];
    }
}

// h -= (sum - target) / count on non-solid nodes
__global__ void ws_eta_shift_kernel(int nn, double* h, const uint8_t* mask, const double* acc, double target)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nn || mask[k] == MACLAB_SOLID || !(acc[1] > 0.0)) return;
    h[k] -= (acc[0] - target) / acc[1];
}

int grid_for(size_t n, int cap = 4096) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, cap)); }

uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

// ===========================================================================
struct maclab_ws_s {
    maclab_ws_config cfg{};
    cudaStream_t stream = nullptr;
    struct Layer {
        int cin, cout, dil, relu_in;
        int64_t w_off, b_off;   // offsets into the parameter vector
        bf16* Wf = nullptr;     // [9][cout][cin]
        bf16* Wb = nullptr;     // [9][cin][cout], flipped
    };
    std::vector<Layer> layers;  // lift, blocks, head
    LayerTable table{};         // the layers for ws_update_kernel
    bf16* Wf_all = nullptr;     // packed weights, each layer's at its parameter offset
    bf16* Wb_all = nullptr;
    int64_t nparam = 0;
    float* param = nullptr;     // master weights
    float* grad = nullptr;
    float* m1 = nullptr;
    float* m2 = nullptr;
    int64_t step = 0;
    bf16* X = nullptr;          // [B][R][R][16]
    std::vector<bf16*> H;       // H_1 .. H_{L+1}, [B][R][R][C]
    bf16* G[2] = {nullptr, nullptr};  // gradient ping-pong [B][R][R][C]
    std::vector<bf16*> GK;      // kept gradients w.r.t. H_1 .. H_{L+1} (maclab_ws_keep_gradients)
    bool keep = false;
    int fwd_batch = 0;          // batch of the last forward pass (0: none yet)
    int grad_batch = 0;         // batch of the last backward pass while keep is on
    int loss_batch = 0;         // batch of the last loss (dY) after the last forward pass
    bf16* dY = nullptr;         // [B][R][R][16]
    float* Yf = nullptr;        // [B][R][R][16]
    double* loss = nullptr;
    double* acc = nullptr;      // decode's (sum of eta, count)
    float* part = nullptr;      // split and block partial sums of the gradients
    double* dpart = nullptr;    // block partials of the loss and of decode's sums
    size_t part_floats = 0;
    int* tc_err = nullptr;      // set when a tensor-core wait timed out
    std::vector<void*> bufs;
    std::string err;
};

namespace {

int wfail(maclab_ws_t w, int code, const std::string& msg)
{
    if (w) w->err = msg;
    maclab_note_error(msg);
    return code;
}

template <typename T>
bool walloc(maclab_ws_t w, T** p, size_t count)
{
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 256)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    w->bufs.push_back(q);
    *p = (T*)q;
    return true;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
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
    return encode;
}

// 4-d map of an NHWC bf16 tensor [batch][R][R][C] with a box of bc
// channels x bx x by pixels; rows of bc channels, swizzled to their width
// (128 bytes for 64 channels, 32 bytes for 16)
bool act_map(CUtensorMap* m, const bf16* p, int C, int R, int batch, int bc, int bx, int by)
{
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)R, (cuuint64_t)R, (cuuint64_t)batch};
    const cuuint64_t str[3] = {(cuuint64_t)C * 2, (cuuint64_t)R * C * 2, (cuuint64_t)R * R * C * 2};
    const cuuint32_t box[4] = {(cuuint32_t)bc, (cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)p, dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  bc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-d map of the packed weights [9 Cout][Cin], box of bc channels x bn rows
bool weight_map(CUtensorMap* m, const bf16* Wk, int Cin, int Cout, int bc, int bn)
{
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Cin, (cuuint64_t)9 * Cout};
    const cuuint64_t str[1] = {(cuuint64_t)Cin * 2};
    const cuuint32_t box[2] = {(cuuint32_t)bc, (cuuint32_t)bn};
    const cuuint32_t one[2] = {1, 1};
    return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)Wk, dims, str, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  bc == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the tcgen05 kernels' configurations: operand buffers (three stages: two
// convolution blocks share an SM) and the weight gradient's blocks
#ifndef MACLAB_T5_CS
#define MACLAB_T5_CS 1
#endif
constexpr int T5_ST = 3, T5_WST = 3;
// blocks of a cluster sharing each weight stage of the 128 -> 128
// convolution by multicast (each fetches 1 / T5_CS of it); 1 by default:
// clusters of 2 and 4 measured slower (forward 0.574 and 0.584 against
// 0.536 ms), the blocks of a cluster waiting for each other's releases
constexpr int T5_CS = MACLAB_T5_CS;
constexpr int T5_WBLOCKS = 150;  // weight-gradient blocks: one per SM, 64 KB stages
template <int KC, int N, int ST>
constexpr size_t t5_conv_smem()
{
    return (size_t)ST * (128 * KC * 2 * (64 / KC) + (64 / KC) * N * KC * 2) + 1024;
}
template <bool MG, int N, int ST>
constexpr size_t t5_wgrad_smem()
{
    return (size_t)ST * ((MG ? 16384 : N * 128) + 3 * (MG ? N * 128 : 16384)) + 1024;
}

// set the dynamic shared-memory limit of every tcgen05 kernel instance
cudaError_t t5_set_limits()
{
    cudaError_t e = cudaFuncSetAttribute(ws_conv5_kernel<64, 128, T5_ST, T5_CS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)t5_conv_smem<64, 128, T5_ST>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_conv5_kernel<16, 128, T5_ST, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)t5_conv_smem<16, 128, T5_ST>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_conv5_kernel<64, 16, T5_ST, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)t5_conv_smem<64, 16, T5_ST>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_wgrad5_kernel<true, 128, T5_WST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)t5_wgrad_smem<true, 128, T5_WST>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_wgrad5_kernel<true, 16, T5_WST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)t5_wgrad_smem<true, 16, T5_WST>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_wgrad5_kernel<false, 16, T5_WST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)t5_wgrad_smem<false, 16, T5_WST>());
    return e;
}

// tensor_path 0: the convolution on ws_conv5_kernel; false if its shape or
// tensor maps are not supported (the caller falls back to mma.sync)
bool launch_conv5(maclab_ws_t w, const ConvArgs& a, int batch)
{
    const int R = a.R;
    const bool shape = (a.Cin % 64 == 0 || a.Cin == 16) && (a.Cout % 128 == 0 || a.Cout == 16) && R % 64 == 0 &&
                       (R < 128 ? 128 % R == 0 : R % 128 == 0);
    if (!shape) return false;
    const int KC = a.Cin == 16 ? 16 : 64, N = a.Cout == 16 ? 16 : 128;
    const int bx = R < 128 ? R : 128, by = 128 / bx;
    const int cs = KC == 64 && N == 128 ? T5_CS : 1;  // the weight box: N / cs rows
    TmaOperands maps;
    if (!act_map(&maps.A, a.X, a.Cin, R, batch, KC, bx, by) || !weight_map(&maps.B, a.Wk, a.Cin, a.Cout, KC, N / cs))
        return false;
    dim3 grid(batch * (R * R / 128), a.Cout / N);
    if (KC == 64 && N == 128 && T5_CS == 1) {
        ws_conv5_kernel<64, 128, T5_ST, 1>
            <<<grid, T5_THREADS, t5_conv_smem<64, 128, T5_ST>(), w->stream>>>(maps, a, w->tc_err);
    } else if (KC == 64 && N == 128) {
        if (grid.x % T5_CS) return false;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(T5_THREADS);
        cfg.dynamicSmemBytes = t5_conv_smem<64, 128, T5_ST>();
        cfg.stream = w->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = T5_CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, ws_conv5_kernel<64, 128, T5_ST, T5_CS>, maps, a, w->tc_err) != cudaSuccess) {
            cudaGetLastError();
            return false;  // the caller falls back to mma.sync
        }
    } else if (KC == 16 && N == 128) {
        ws_conv5_kernel<16, 128, T5_ST, 1>
            <<<grid, T5_THREADS, t5_conv_smem<16, 128, T5_ST>(), w->stream>>>(maps, a, w->tc_err);
    } else if (KC == 64 && N == 16) {
        ws_conv5_kernel<64, 16, T5_ST, 1>
            <<<grid, T5_THREADS, t5_conv_smem<64, 16, T5_ST>(), w->stream>>>(maps, a, w->tc_err);
    } else {
        return false;  // 16 -> 16 channels: no such layer
    }
    return true;
}

void launch_conv(maclab_ws_t w, const ConvArgs& a, int batch)
{
    const int segs = a.R / CONV_M;
    if (w->cfg.tensor_path == 0 && launch_conv5(w, a, batch)) return;
    if (w->cfg.tensor_path == 1 && a.Cin % TC_KS == 0 && a.Cout % TC_N == 0 && (a.R * a.R) % TC_M == 0) {
        dim3 grid(batch * (a.R * a.R / TC_M), a.Cout / TC_N);
        ws_conv_tc_kernel<<<grid, TC_THREADS, TC_SMEM, w->stream>>>(a, w->tc_err);
    } else if (a.Cout % 128 == 0) {
        dim3 grid(batch * a.R * segs, a.Cout / 128);
        ws_conv_kernel<128><<<grid, THREADS, 0, w->stream>>>(a);
    } else {
        dim3 grid(batch * a.R * segs, a.Cout / 16);
        ws_conv_kernel<16><<<grid, THREADS, 0, w->stream>>>(a);
    }
}

// tensor_path 0: the weight gradient on ws_wgrad5_kernel; false if its
// shape or tensor maps are not supported
bool launch_wgrad5(maclab_ws_t w, const WgradArgs& a0)
{
    WgradArgs a = a0;
    const bool mg = a.Cout % 128 == 0 && (a.Cin % 128 == 0 || a.Cin == 16);
    const bool head = !mg && a.Cin % 128 == 0 && a.Cout == 16;
    if (!(mg || head) || a.R % 64) return false;
    const int N = mg ? (a.Cin == 16 ? 16 : 128) : 16;
    const int gbox = (mg || N == 128) ? 64 : 16, xbox = (!mg || N == 128) ? 64 : 16;
    TmaOperands maps;
    if (!act_map(&maps.A, a.dY, a.Cout, a.R, a.B, gbox, 64, 1) || !act_map(&maps.B, a.X, a.Cin, a.R, a.B, xbox, 64, 1))
        return false;
    const int tiles = (mg ? a.Cout / 128 * (a.Cin / N) : a.Cin / 128 * (a.Cout / N));
    const int segs = a.B * a.R * (a.R / 64);
    a.splits = std::max(1, std::min(segs, T5_WBLOCKS / (3 * tiles)));
    a.part = w->part;
    dim3 grid(3, a.splits, tiles);
    if (mg && N == 128)
        ws_wgrad5_kernel<true, 128, T5_WST>
            <<<grid, T5_THREADS, t5_wgrad_smem<true, 128, T5_WST>(), w->stream>>>(maps, a, w->tc_err);
    else if (mg)
        ws_wgrad5_kernel<true, 16, T5_WST>
            <<<grid, T5_THREADS, t5_wgrad_smem<true, 16, T5_WST>(), w->stream>>>(maps, a, w->tc_err);
    else
        ws_wgrad5_kernel<false, 16, T5_WST>
            <<<grid, T5_THREADS, t5_wgrad_smem<false, 16, T5_WST>(), w->stream>>>(maps, a, w->tc_err);
    const size_t n = (size_t)9 * a.Cout * a.Cin;
    ws_sum_parts_kernel<<<grid_for(n), 256, 0, w->stream>>>(w->part, a.splits, n, a.dW);
    return true;
}

void launch_wgrad(maclab_ws_t w, const WgradArgs& a0)
{
    if (w->cfg.tensor_path == 0 && launch_wgrad5(w, a0)) return;
    WgradArgs a = a0;
    const int chunks = a.B * a.R * a.R / WG_K;
    const int MT = a.Cout % 64 == 0 ? 64 : 16, NT = a.Cin % 64 == 0 ? 64 : 16;
    const int tiles = (a.Cout / MT) * (a.Cin / NT);
    // about two blocks per SM over all (tile, tap, split) blocks
    a.splits = std::max(1, std::min(chunks, 304 / std::max(1, tiles * 9) + 1));
    a.part = w->part;
    dim3 grid(tiles, 9, a.splits);
    if (MT == 64 && NT == 64) ws_wgrad_kernel<64, 64><<<grid, THREADS, 0, w->stream>>>(a);
    else if (MT == 64) ws_wgrad_kernel<64, 16><<<grid, THREADS, 0, w->stream>>>(a);
    else ws_wgrad_kernel<16, 64><<<grid, THREADS, 0, w->stream>>>(a);
    const size_t n = (size_t)9 * a.Cout * a.Cin;
    ws_sum_parts_kernel<<<grid_for(n), 256, 0, w->stream>>>(w->part, a.splits, n, a.dW);
}

// Floats of the partial-sum buffer: the weight gradient's splits of every
// layer (at most 304 / (tiles * 9) + 1 of them on mma.sync, T5_WBLOCKS / 3
// on tcgen05) and the bias gradient's block rows.
size_t part_floats_for(const maclab_ws_s* w)
{
    size_t n = 0;
    for (const auto& L : w->layers) {
        const int MT = L.cout % 64 == 0 ? 64 : 16, NT = L.cin % 64 == 0 ? 64 : 16;
        const int tiles = (L.cout / MT) * (L.cin / NT);
        const size_t S = (size_t)(304 / std::max(1, tiles * 9) + 1);
        n = std::max(n, std::max(S, (size_t)(T5_WBLOCKS / 3)) * 9 * L.cout * L.cin);
        n = std::max(n, (size_t)BG_BLOCKS * L.cout);
    }
    return n;
}

// pack the weights (and with lr_t > 0 first take one Adam step)
void update(maclab_ws_t w, int adam, float lr_t)
{
    ws_update_kernel<<<grid_for((size_t)w->nparam), 256, 0, w->stream>>>(
        w->param, w->grad, w->m1, w->m2, (size_t)w->nparam, adam, lr_t, 0.9f, 0.999f, 1e-8f, w->table, w->Wf_all,
        w->Wb_all);
}

// forward of `batch` samples from w->X; head output to w->Yf
void forward(maclab_ws_t w, int batch)
{
    const int R = w->cfg.res;
    const int nl = (int)w->layers.size();
    const bf16* in = w->X;
    for (int l = 0; l < nl; ++l) {
        const auto& L = w->layers[l];
        ConvArgs a{};
        a.X = in;
        a.Wk = L.Wf;
        a.bias = w->param + L.b_off;
        a.R = R;
        a.Cin = L.cin;
        a.Cout = L.cout;
        a.dil = L.dil;
        a.relu_in = L.relu_in;
        if (l == nl - 1) {
            a.Yf = w->Yf;
        } else {
            a.Y = w->H[l];
            if (l > 0) a.res = w->H[l - 1];  // residual block
        }
        launch_conv(w, a, batch);
        if (l < nl - 1) in = w->H[l];
    }
    w->fwd_batch = batch;
    w->loss_batch = w->grad_batch = 0;
}

// gradients of the loss into w->grad (zeroed first); dY from the loss kernel
void backward(maclab_ws_t w, int batch)
{
    const int R = w->cfg.res;
    const int nl = (int)w->layers.size();
    const int P = batch * R * R;
    cudaMemsetAsync(w->grad, 0, (size_t)w->nparam * sizeof(float), w->stream);
    const bf16* gout = w->dY;  // gradient w.r.t. the output of layer l
    int ping = 0;
    for (int l = nl - 1; l >= 0; --l) {
        const auto& L = w->layers[l];
        const bf16* xin = l == 0 ? w->X : w->H[l - 1];
        WgradArgs g{};
        g.dY = gout;
        g.X = xin;
        g.dW = w->grad + L.w_off;
        g.B = batch;
        g.R = R;
        g.Cin = L.cin;
        g.Cout = L.cout;
        g.dil = L.dil;
        g.relu_in = L.relu_in;
        launch_wgrad(w, g);
        ws_bias_grad_kernel<<<BG_BLOCKS, THREADS, 0, w->stream>>>(gout, P, L.cout, w->part);
        ws_sum_parts_kernel<<<grid_for(L.cout), 256, 0, w->stream>>>(w->part, BG_BLOCKS, L.cout, w->grad + L.b_off);
        if (l == 0) break;
        // gradient w.r.t. this layer's input H_{l-1}:
        //   head:  relu'(H) * conv^T(gout)
        //   block: gout + relu'(H) * conv^T(gout)
        ConvArgs a{};
        a.X = gout;
        a.Wk = L.Wb;
        a.R = R;
        a.Cin = L.cout;
        a.Cout = L.cin;
        a.dil = L.dil;
        a.relu_in = 0;
        a.gate = w->H[l - 1];
        a.res = l < nl - 1 ? gout : nullptr;
        a.Y = w->keep ? w->GK[l - 1] : w->G[ping];
        launch_conv(w, a, batch);
        gout = a.Y;
        ping ^= 1;
    }
    w->grad_batch = w->keep ? batch : 0;
}

int check_batch(maclab_ws_t w, int batch)
{
    if (!w) return wfail(nullptr, MACLAB_E_ARG, "NULL warm-start handle");
    if (batch < 1 || batch > w->cfg.max_batch) return wfail(w, MACLAB_E_ARG, "batch must be 1..max_batch");
    return MACLAB_OK;
}

int loss_and_grad(maclab_ws_t w, int batch, int oc, const float* x, const float* t, const float* wt)
{
    const int R = w->cfg.res;
    const size_t P = (size_t)batch * R * R;
    ws_to_bf16_kernel<<<grid_for(P * IO), 256, 0, w->stream>>>(x, w->X, P * IO);
    forward(w, batch);
    const int nb = grid_for(P * IO, 1024);
    ws_loss_kernel<<<nb, THREADS, 0, w->stream>>>(w->Yf, t, wt, (int)P, oc, w->dY, w->dpart);
    ws_sum_doubles_kernel<<<1, THREADS, 0, w->stream>>>(w->dpart, nb, 1, w->loss);
    w->loss_batch = batch;
    backward(w, batch);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("warm-start launch: ") + cudaGetErrorString(e));
    return MACLAB_OK;
}

int check_tc(maclab_ws_t w)
{
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, w->tc_err, sizeof(int), cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("warm-start status: ") + cudaGetErrorString(e));
    if (flag) return wfail(w, MACLAB_E_CUDA, "warm start: a tensor-core wait timed out");
    return MACLAB_OK;
}

int read_loss(maclab_ws_t w, double* loss)
{
    if (!loss) return MACLAB_OK;
    cudaError_t e = cudaMemcpyAsync(loss, w->loss, sizeof(double), cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("warm-start loss: ") + cudaGetErrorString(e));
    return check_tc(w);
}

}  // namespace

extern "C" {

int maclab_ws_create(const maclab_ws_config* cfg, void* stream, maclab_ws_t* out)
{
    if (!cfg || !out) return wfail(nullptr, MACLAB_E_ARG, "NULL argument");
    *out = nullptr;
    if (cfg->res < 64 || cfg->res % 64 || cfg->channels < 64 || cfg->channels % 64 || cfg->blocks < 0 ||
        cfg->blocks > 64 || cfg->max_batch < 1)
        return wfail(nullptr, MACLAB_E_ARG, "need res and channels multiples of 64, 0 <= blocks <= 64, max_batch >= 1");
    if (cfg->tensor_path < 0 || cfg->tensor_path > 2)
        return wfail(nullptr, MACLAB_E_ARG, "tensor_path must be 0, 1 or 2");
    for (int l = 0; l < cfg->blocks; ++l)
        if (cfg->dilation[l] < 1 || cfg->dilation[l] >= cfg->res)
            return wfail(nullptr, MACLAB_E_ARG, "dilations must be in 1..res-1");
    maclab_ws_t w = new maclab_ws_s;
    w->cfg = *cfg;
    w->stream = (cudaStream_t)stream;
    const int C = cfg->channels, R = cfg->res;
    auto add = [&](int cin, int cout, int dil, int relu) {
        maclab_ws_s::Layer L;
        L.cin = cin;
        L.cout = cout;
        L.dil = dil;
        L.relu_in = relu;
        L.w_off = w->nparam;
        w->nparam += (int64_t)9 * cin * cout;
        L.b_off = w->nparam;
        w->nparam += cout;
        w->layers.push_back(L);
    };
    add(IO, C, 1, 0);
    for (int l = 0; l < cfg->blocks; ++l) add(C, C, cfg->dilation[l], 1);
    add(C, IO, 1, 1);
    const size_t P = (size_t)cfg->max_batch * R * R;
    bool ok = walloc(w, &w->param, w->nparam) && walloc(w, &w->grad, w->nparam) && walloc(w, &w->m1, w->nparam) &&
              walloc(w, &w->m2, w->nparam) && walloc(w, &w->X, P * IO) && walloc(w, &w->dY, P * IO) &&
              walloc(w, &w->Yf, P * IO) && walloc(w, &w->loss, 1) && walloc(w, &w->acc, 2) && walloc(w, &w->tc_err, 1) && walloc(w, &w->G[0], P * C) &&
              walloc(w, &w->G[1], P * C);
    w->part_floats = part_floats_for(w);
    ok = ok && walloc(w, &w->part, w->part_floats) && walloc(w, &w->dpart, 2 * 1024);
    w->H.assign(w->layers.size() - 1, nullptr);
    for (size_t l = 0; ok && l < w->H.size(); ++l) ok = walloc(w, &w->H[l], P * C);
    ok = ok && walloc(w, &w->Wf_all, w->nparam) && walloc(w, &w->Wb_all, w->nparam);
    w->table.n = (int)w->layers.size();
    for (int l = 0; ok && l < w->table.n; ++l) {
        auto& L = w->layers[l];
        L.Wf = w->Wf_all + L.w_off;
        L.Wb = w->Wb_all + L.w_off;
        w->table.w_off[l] = L.w_off;
        w->table.cin[l] = L.cin;
        w->table.cout[l] = L.cout;
    }
    if (!ok) {
        maclab_ws_destroy(w);
        return wfail(nullptr, MACLAB_E_NOMEM, "warm-start device allocation failed");
    }
    // initial weights: normal(0, sqrt(2 / fan_in)) by Box-Muller on SplitMix64;
    // the residual branches start small and the head at zero
    std::vector<float> h(w->nparam, 0.f);
    uint64_t s = cfg->seed;
    for (size_t li = 0; li < w->layers.size(); ++li) {
        const auto& L = w->layers[li];
        const bool head = li + 1 == w->layers.size();
        const double sd = head ? 0.0 : std::sqrt(2.0 / (9.0 * L.cin)) * (li == 0 ? 1.0 : 0.2);
        for (int64_t k = 0; k < (int64_t)9 * L.cin * L.cout; ++k) {
            const double u1 = ((splitmix(s) >> 11) + 1) * (1.0 / 9007199254740993.0);
            const double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
            h[L.w_off + k] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    cudaError_t e = cudaMemcpyAsync(w->param, h.data(), h.size() * 4, cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->m1, 0, (size_t)w->nparam * 4, w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->m2, 0, (size_t)w->nparam * 4, w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->tc_err, 0, sizeof(int), w->stream);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ws_conv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    if (e == cudaSuccess) e = t5_set_limits();
    if (e == cudaSuccess) {
        update(w, 0, 0.f);
        e = cudaStreamSynchronize(w->stream);
    }
    if (e != cudaSuccess) {
        maclab_ws_destroy(w);
        return wfail(nullptr, MACLAB_E_CUDA, std::string("warm-start init: ") + cudaGetErrorString(e));
    }
    *out = w;
    return MACLAB_OK;
}

void maclab_ws_destroy(maclab_ws_t w)
{
    if (!w) return;
    cudaStreamSynchronize(w->stream);
    for (void* p : w->bufs) cudaFree(p);
    delete w;
}

int maclab_ws_param_count(maclab_ws_t w, int64_t* n)
{
    if (!w || !n) return wfail(w, MACLAB_E_ARG, "NULL argument");
    *n = w->nparam;
    return MACLAB_OK;
}

int maclab_ws_get_params(maclab_ws_t w, float* host, int64_t n)
{
    if (!w || !host || n != w->nparam) return wfail(w, MACLAB_E_ARG, "need the handle's parameter count");
    cudaError_t e = cudaMemcpyAsync(host, w->param, n * 4, cudaMemcpyDeviceToHost, w->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("get_params: ") + cudaGetErrorString(e));
    return MACLAB_OK;
}

int maclab_ws_set_params(maclab_ws_t w, const float* host, int64_t n)
{
    if (!w || !host || n != w->nparam) return wfail(w, MACLAB_E_ARG, "need the handle's parameter count");
    cudaError_t e = cudaMemcpyAsync(w->param, host, n * 4, cudaMemcpyHostToDevice, w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->m1, 0, (size_t)n * 4, w->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->m2, 0, (size_t)n * 4, w->stream);
    if (e == cudaSuccess) {
        update(w, 0, 0.f);
        e = cudaStreamSynchronize(w->stream);
    }
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("set_params: ") + cudaGetErrorString(e));
    w->step = 0;
    return MACLAB_OK;
}

int maclab_ws_forward(maclab_ws_t w, int batch, const float* x, float* y)
{
    int rc = check_batch(w, batch);
    if (rc != MACLAB_OK) return rc;
    if (!x || !y) return wfail(w, MACLAB_E_ARG, "NULL tensor");
    const int R = w->cfg.res;
    const size_t P = (size_t)batch * R * R;
    ws_to_bf16_kernel<<<grid_for(P * IO), 256, 0, w->stream>>>(x, w->X, P * IO);
    forward(w, batch);
    cudaError_t e = cudaMemcpyAsync(y, w->Yf, P * IO * 4, cudaMemcpyDeviceToDevice, w->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("warm-start forward: ") + cudaGetErrorString(e));
    return MACLAB_OK;
}

int maclab_ws_gradients(maclab_ws_t w, int batch, int oc, const float* x, const float* t, const float* wt,
                        float* grad_host, int64_t n, double* loss)
{
    int rc = check_batch(w, batch);
    if (rc != MACLAB_OK) return rc;
    if (!x || !t || !wt || !grad_host || n != w->nparam || oc < 1 || oc > IO)
        return wfail(w, MACLAB_E_ARG, "NULL tensor, wrong parameter count or out_ch");
    if ((rc = loss_and_grad(w, batch, oc, x, t, wt)) != MACLAB_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(grad_host, w->grad, n * 4, cudaMemcpyDeviceToHost, w->stream);
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("gradients: ") + cudaGetErrorString(e));
    if (loss) return read_loss(w, loss);
    return check_tc(w);
}

int maclab_ws_train_step(maclab_ws_t w, int batch, int oc, const float* x, const float* t, const float* wt, float lr,
                         double* loss)
{
    int rc = check_batch(w, batch);
    if (rc != MACLAB_OK) return rc;
    if (!x || !t || !wt || oc < 1 || oc > IO || !(lr >= 0.f)) return wfail(w, MACLAB_E_ARG, "bad train_step argument");
    if ((rc = loss_and_grad(w, batch, oc, x, t, wt)) != MACLAB_OK) return rc;
    w->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const double lr_t = lr * std::sqrt(1.0 - std::pow(b2, (double)w->step)) / (1.0 - std::pow(b1, (double)w->step));
    update(w, 1, (float)lr_t);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("train_step: ") + cudaGetErrorString(e));
    return read_loss(w, loss);
}

int maclab_ws_keep_gradients(maclab_ws_t w, int on)
{
    if (!w) return wfail(nullptr, MACLAB_E_ARG, "NULL warm-start handle");
    if (on && w->GK.empty()) {
        const size_t P = (size_t)w->cfg.max_batch * w->cfg.res * w->cfg.res;
        std::vector<bf16*> k(w->H.size(), nullptr);
        for (auto& p : k)
            if (!walloc(w, &p, P * w->cfg.channels)) return wfail(w, MACLAB_E_NOMEM, "keep_gradients: out of memory");
        w->GK = k;
    }
    w->keep = on != 0;
    w->grad_batch = 0;
    return MACLAB_OK;
}

int maclab_ws_inspect(maclab_ws_t w, int what, int index, int batch, float* out, int64_t n)
{
    if (!w || !out) return wfail(w, MACLAB_E_ARG, "NULL argument");
    const int L1 = (int)w->H.size();
    const size_t pix = (size_t)batch * w->cfg.res * w->cfg.res;
    const bf16* src = nullptr;
    const float* srcf = nullptr;
    size_t ch = w->cfg.channels;
    if (what == 0 || what == 1) {
        if (index < 0 || index >= L1) return wfail(w, MACLAB_E_ARG, "inspect: index must be 0..blocks");
        if (what == 0 && (batch < 1 || batch > w->fwd_batch))
            return wfail(w, MACLAB_E_ARG, "inspect: batch exceeds the last forward pass");
        if (what == 1 && (batch < 1 || batch > w->grad_batch))
            return wfail(w, MACLAB_E_ARG, "inspect: no kept gradients of that batch");
        src = what == 0 ? w->H[index] : w->GK[index];
    } else if (what == 2 || what == 3) {
        if (index != 0) return wfail(w, MACLAB_E_ARG, "inspect: index must be 0");
        if (batch < 1 || batch > (what == 2 ? w->loss_batch : w->fwd_batch))
            return wfail(w, MACLAB_E_ARG, "inspect: batch exceeds the last pass");
        ch = IO;
        if (what == 2) src = w->dY;
        else srcf = w->Yf;
    } else {
        return wfail(w, MACLAB_E_ARG, "inspect: what must be 0..3");
    }
    if (n != (int64_t)(pix * ch)) return wfail(w, MACLAB_E_ARG, "inspect: n must be batch * res * res * channels");
    cudaError_t e = cudaSuccess;
    if (src) ws_from_bf16_kernel<<<grid_for(pix * ch), 256, 0, w->stream>>>(src, out, pix * ch);
    else e = cudaMemcpyAsync(out, srcf, pix * ch * 4, cudaMemcpyDeviceToDevice, w->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("inspect: ") + cudaGetErrorString(e));
    return MACLAB_OK;
}

int maclab_ws_encode(maclab_ws_t w, int n, const float* D, const uint8_t* mask, double wind_u, double wind_v,
                     double Cb, double dx, const float* eta, const float* u, const float* v, int pitch, const double scale[4],
                     float* x, float* t, float* wt)
{
    if (!w || !D || !mask || !scale || !x) return wfail(w, MACLAB_E_ARG, "NULL argument");
    if (!(dx > 0)) return wfail(w, MACLAB_E_ARG, "dx must be positive");
    const int R = w->cfg.res;
    if (n != R * CELL) return wfail(w, MACLAB_E_ARG, "fine grid must be res * MACLAB_WS_CELL per side");
    if (eta && (!u || !v || !t || !wt || pitch < n)) return wfail(w, MACLAB_E_ARG, "state needs u, v, targets, pitch");
    for (int k = 0; k < 4; ++k)
        if (!(scale[k] > 0)) return wfail(w, MACLAB_E_ARG, "scales must be positive");
    ws_encode_kernel<<<(R * R + 255) / 256, 256, 0, w->stream>>>(n, R, D, mask, (float)wind_u, (float)wind_v,
                                                                 (float)Cb, (float)dx, eta, u, v, pitch, (float)scale[0],
                                                                 (float)scale[1], (float)scale[2], (float)scale[3], x,
                                                                 eta ? t : nullptr, wt);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("encode: ") + cudaGetErrorString(e));
    return MACLAB_OK;
}

int maclab_ws_decode(maclab_ws_t w, int n, const float* y, const float* D, const uint8_t* mask, const double scale[4],
                     double mass_eta, double* h, double* u, double* v)
{
    if (!w || !y || !D || !mask || !scale || !h || !u || !v) return wfail(w, MACLAB_E_ARG, "NULL argument");
    const int R = w->cfg.res;
    if (n != R * CELL) return wfail(w, MACLAB_E_ARG, "fine grid must be res * MACLAB_WS_CELL per side");
    ws_decode_kernel<<<(n * n + 255) / 256, 256, 0, w->stream>>>(n, R, y, D, mask, scale[1], scale[2], scale[3], h,
                                                                 u, v);
    if (std::isfinite(mass_eta)) {
        const int nb = grid_for((size_t)n * n, 1024);
        ws_eta_sum_kernel<<<nb, THREADS, 0, w->stream>>>(n * n, h, D, mask, w->dpart);
        ws_sum_doubles_kernel<<<2, THREADS, 0, w->stream>>>(w->dpart, nb, 2, w->acc);
        ws_eta_shift_kernel<<<(n * n + 255) / 256, 256, 0, w->stream>>>(n * n, h, mask, w->acc, mass_eta);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return wfail(w, MACLAB_E_CUDA, std::string("decode: ") + cudaGetErrorString(e));
    return MACLAB_OK;
}

}  // extern "C"
