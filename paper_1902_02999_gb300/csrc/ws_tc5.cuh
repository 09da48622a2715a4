// ws_tc5.cuh -- the warm-start network's convolutions (forward and input
// gradient) and weight gradients on tcgen05.mma, operands brought in by TMA
// tensor copies, accumulators in tensor memory.  Included by warmstart.cu
// inside its anonymous namespace (uses its ConvArgs, WgradArgs, relu2,
// smem_addr and mbarrier helpers).
//
// Both kernels split a block's 6 warps by role, each role waiting only on
// the mbarriers it needs (no block barrier in the main loop):
//   warp 0, lane 0   issues the tensor copies of a stage once the MMAs that
//                    last read its buffer have completed ("empty");
//   warp 1, lane 0   issues the stage's MMAs once its operands are in
//                    ("full", or "ready" after rectification) and commits
//                    them to the buffer's "empty" barrier;
//   warps 2..5       rectify the stage's activation operand in shared
//                    memory when the layer's input is relu(H) (then arrive on
//                    "ready"), and afterwards read the accumulators out of
//                    tensor memory (warp w owns lanes 32 (w mod 4) ..) for
//                    the epilogue.
// Other lanes of warps 0 and 1 wait at a warp barrier, never spinning on an
// mbarrier beside the lane that issues.  Every wait is bounded: on time-out
// the block records it in *err, lets the copies in flight land (bounded)
// and leaves without writing its outputs.

constexpr int T5_THREADS = 192;
constexpr uint32_t T5_SW128 = 2, T5_SW32 = 6;  // descriptor swizzle modes: 128-byte and 32-byte

// shared-memory matrix descriptor: start, leading and stride byte offsets,
// descriptor version 1 at bit 46, swizzle mode at bit 61
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t mode)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)mode << 61;
    return d;
}

// instruction descriptor, kind::f16: f32 accumulate, bf16 A and B; bit 15
// (16) set when A (B) is MN-major instead of K-major; N >> 3 at bit 17,
// M >> 4 at bit 24
__host__ __device__ constexpr uint32_t t5_idesc(int M, int N, bool a_mn, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__host__ __device__ constexpr uint32_t t5_cols(int n)
{
    return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512;
}

__device__ __forceinline__ void t5_bar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void t5_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void t5_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// lane 0 waits (bounded), the warp learns the outcome
__device__ __forceinline__ bool t5_warp_wait(uint32_t bar, uint32_t parity, int lane)
{
    bool ok = true;
    if (lane == 0) ok = tc_mbar_wait(bar, parity);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
__device__ __forceinline__ void t5_load4(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                         uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void t5_load2(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
// the same copy delivered to the same offset, and signalled on the same
// barrier, in every block of the cluster named in mask
__device__ __forceinline__ void t5_load2_mc(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar,
                                            uint16_t mask)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1, {%2, "
        "%3}], [%4], %5;\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar), "h"(mask)
        : "memory");
}
__device__ __forceinline__ uint32_t t5_cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ void t5_cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void t5_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void t5_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}
// arrives, once the MMAs complete, on the barrier at this offset in every
// block of the cluster named in mask
__device__ __forceinline__ void t5_commit_mc(uint32_t bar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n" ::
                     "r"(bar),
                 "h"(mask)
                 : "memory");
}
// relu of `bytes` bytes of bf16 pairs, by nt threads (t = 0 .. nt-1)
__device__ __forceinline__ void t5_rectify(unsigned char* p, uint32_t bytes, int t, int nt)
{
    for (uint32_t i = (uint32_t)t * 16u; i < bytes; i += (uint32_t)nt * 16u) {
        uint4* q = reinterpret_cast<uint4*>(p + i);
        uint4 v = *q;
        v.x = relu2(v.x);
        v.y = relu2(v.y);
        v.z = relu2(v.z);
        v.w = relu2(v.w);
        *q = v;
    }
}
__device__ __forceinline__ void t5_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Block start-up shared by both kernels: tensor memory (warp 0) and the
// barriers (thread 0); full and empty count one arrival, ready four (the
// rectifying warps), done one.
template <int ST>
struct T5Bars {
    uint64_t full[ST], ready[ST], empty[ST], done;
};
template <int ST, int CS = 1>
__device__ __forceinline__ uint32_t t5_start(T5Bars<ST>& bars, uint32_t* tmem_slot, uint32_t cols, int* flags)
{
    const int tid = threadIdx.x;
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(tmem_slot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < ST; ++k) {
            t5_bar_init(smem_addr(&bars.full[k]), 1);
            t5_bar_init(smem_addr(&bars.ready[k]), 4);
            t5_bar_init(smem_addr(&bars.empty[k]), CS);  // every block of the cluster releases it
        }
        t5_bar_init(smem_addr(&bars.done), 1);
        flags[0] = flags[1] = flags[2] = 0;  // abort, stages issued, stages seen landed
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    if (CS > 1)
        t5_cluster_sync();  // no block copies into a peer's buffers before its barriers exist
    else
        __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    return *tmem_slot;
}
// Block end: after a time-out, the copies still in flight land (bounded)
// before shared and tensor memory are released.
template <int ST, int CS = 1>
__device__ __forceinline__ void t5_finish(T5Bars<ST>& bars, uint32_t tmem, uint32_t cols, int* flags, int* err)
{
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && flags[0]) {
        for (int s = flags[2]; s < flags[1]; ++s) tc_mbar_wait(smem_addr(&bars.full[s % ST]), (uint32_t)(s / ST) & 1u);
        atomicOr(err, 1);
    }
    // with a cluster: no block leaves while a peer's copies or MMA
    // completions may still signal its barriers (every peer has waited for
    // its own MMAs by now)
    if (CS > 1)
        t5_cluster_sync();
    else
        __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(cols) : "memory");
}

// ---------------------------------------------------------------------------
// Convolution (forward, or input gradient with a gate): a block owns a
// tile of 128 consecutive pixels of an image (M = 128) and N output
// channels; K runs over 9 taps x C_in in chunks of KC channels of one tap,
// 64 / KC chunks a stage.  KC = 64: rows of 128 bytes, 128-byte swizzle;
// KC = 16 (16-channel input): rows of 32 bytes, 32-byte swizzle.  Both
// operands K-major; A = the activations at the tap's offset (zero fill
// outside the image), B = the weights [9 C_out][C_in].  The epilogue warps
// load the bias into shared memory and their pixel's residual row and gate
// signs into registers before the main loop, so that only the accumulator
// is waited for at the end.
//   stage layout: A chunks [64 / KC] of 128 x KC bf16, then B chunks
//   [64 / KC] of N x KC bf16, every chunk on a 1024-byte boundary.
template <int KC, int N, int ST, int CS>
__global__ void __launch_bounds__(T5_THREADS, 2) ws_conv5_kernel(const __grid_constant__ TmaOperands maps,
                                                               const ConvArgs a, int* err)
{
    constexpr uint16_t MASK = (uint16_t)((1u << CS) - 1u);
    constexpr int CPS = 64 / KC;
    constexpr uint32_t ACH = 128 * KC * 2, BCH = N * KC * 2;
    constexpr uint32_t ABYTES = CPS * ACH, SBYTES = ABYTES + CPS * BCH;
    constexpr uint32_t MODE = KC == 64 ? T5_SW128 : T5_SW32, SBO = KC == 64 ? 1024 : 256;
    constexpr uint32_t IDESC = t5_idesc(128, N, false, false);
    constexpr uint32_t COLS = t5_cols(N);
    extern __shared__ __align__(16) unsigned char t5_raw[];
    __shared__ __align__(8) T5Bars<ST> bars;
    __shared__ uint32_t tmem_slot;
    __shared__ int flags[3];
    __shared__ float sbias[N];
    const uint32_t raw = smem_addr(t5_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* tsm = t5_raw + (base - raw);
    const int R = a.R, Cin = a.Cin, Cout = a.Cout, dil = a.dil;
    const int P = R * R, tiles = P / 128;
    const int b = blockIdx.x / tiles, p0 = (blockIdx.x % tiles) * 128;
    const int n0 = blockIdx.y * N;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kch = Cin / KC, KT = 9 * kch, NS = (KT + CPS - 1) / CPS;
    const uint32_t tmem = t5_start<ST, CS>(bars, &tmem_slot, COLS, flags);
    const int rank = CS > 1 ? (int)t5_cluster_rank() : 0;

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            for (; s < NS; ++s) {
                const int buf = s % ST;
                if (s >= ST && !tc_mbar_wait(smem_addr(&bars.empty[buf]), (uint32_t)(s / ST + 1) & 1u)) {
                    atomicOr(&flags[0], 1);
                    break;
                }
                const int c0 = s * CPS, nc = min(CPS, KT - c0);
                const uint32_t sA = base + buf * SBYTES, sB = sA + ABYTES, bar = smem_addr(&bars.full[buf]);
                // the block's own A; B whole, of which this block fetches
                // rows [rank N / CS, (rank + 1) N / CS) for every block of
                // the cluster (the clusters' blocks share n0)
                t5_expect(bar, (uint32_t)nc * (ACH + BCH));
                for (int c = 0; c < nc; ++c) {
                    const int kk = c0 + c, tap = kk / kch, ci0 = (kk % kch) * KC;
                    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                    t5_load4(sA + c * ACH, &maps.A, ci0, p0 % R + dx * dil, p0 / R + dy * dil, b, bar);
                    if (CS > 1)
                        t5_load2_mc(sB + c * BCH + rank * (BCH / CS), &maps.B, ci0, tap * Cout + n0 + rank * (N / CS),
                                    bar, MASK);
                    else
                        t5_load2(sB + c * BCH, &maps.B, ci0, tap * Cout + n0, bar);
                }
            }
            flags[1] = s;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            for (; s < NS; ++s) {
                const int buf = s % ST;
                const uint32_t bar = smem_addr(a.relu_in ? &bars.ready[buf] : &bars.full[buf]);
                if (!tc_mbar_wait(bar, (uint32_t)(s / ST) & 1u)) {
                    atomicOr(&flags[0], 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const int c0 = s * CPS, nc = min(CPS, KT - c0);
                const uint32_t sA = base + buf * SBYTES, sB = sA + ABYTES;
                for (int c = 0; c < nc; ++c) {
#pragma unroll
                    for (int k16 = 0; k16 < KC / 16; ++k16) {
                        const uint64_t ad = t5_desc(sA + c * ACH + k16 * 32, 16, SBO, MODE);
                        const uint64_t bd = t5_desc(sB + c * BCH + k16 * 32, 16, SBO, MODE);
                        t5_mma(tmem, ad, bd, IDESC, (s | c | k16) != 0 ? 1u : 0u);
                    }
                }
                // the buffer is free once every block of the cluster is done
                // with it (its B arrived in all of them together)
                if (CS > 1)
                    t5_commit_mc(smem_addr(&bars.empty[buf]), MASK);
                else
                    t5_commit(smem_addr(&bars.empty[buf]));
            }
            if (!a.relu_in) flags[2] = s;
            // arrives once every MMA issued above has completed
            t5_commit(smem_addr(&bars.done));
        }
        __syncwarp();
    } else {
        // before the main loop: bias to shared memory, this lane's pixel's
        // residual row and gate signs to registers
        const int q = warp & 3;  // tensor-memory lanes 32 q .. 32 q + 31
        const int m = q * 32 + lane;
        const size_t o0 = ((size_t)b * P + p0 + m) * Cout + n0;
        for (int c = tid - 64; c < N; c += T5_THREADS - 64) sbias[c] = a.bias ? a.bias[n0 + c] : 0.f;
        uint4 rres[N / 8];
        uint32_t gbits[(N + 31) / 32];
#pragma unroll
        for (int k = 0; k < N / 8; ++k) rres[k] = a.res ? reinterpret_cast<const uint4*>(a.res + o0)[k] : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < (N + 31) / 32; ++k) gbits[k] = 0xFFFFFFFFu;
        if (a.gate) {
#pragma unroll
            for (int k = 0; k < N / 8; ++k) {
                const uint4 g4 = reinterpret_cast<const uint4*>(a.gate + o0)[k];
                const __nv_bfloat162* gt = reinterpret_cast<const __nv_bfloat162*>(&g4);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int c = 8 * k + 2 * j;
                    if (!(__bfloat162float(gt[j].x) > 0.f)) gbits[c >> 5] &= ~(1u << (c & 31));
                    if (!(__bfloat162float(gt[j].y) > 0.f)) gbits[(c + 1) >> 5] &= ~(1u << ((c + 1) & 31));
                }
            }
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");  // sbias written by the four epilogue warps
        if (a.relu_in) {
            int s = 0;
            for (; s < NS; ++s) {
                const int buf = s % ST;
                if (!t5_warp_wait(smem_addr(&bars.full[buf]), (uint32_t)(s / ST) & 1u, lane)) {
                    if (lane == 0) atomicOr(&flags[0], 1);
                    break;
                }
                t5_rectify(tsm + buf * SBYTES, ABYTES, tid - 64, T5_THREADS - 64);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) t5_arrive(smem_addr(&bars.ready[buf]));
            }
            if (warp == 2 && lane == 0) flags[2] = s;
        }
        const bool fin = t5_warp_wait(smem_addr(&bars.done), 0, lane);
        if (!fin && lane == 0) atomicOr(&flags[0], 1);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (fin && !*(volatile int*)&flags[0]) {
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t r[16];
                t5_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
                const size_t o = o0 + c0;
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(r[j]) + sbias[c0 + j];
                    if (!((gbits[(c0 + j) >> 5] >> ((c0 + j) & 31)) & 1u)) v[j] = 0.f;
                }
                if (a.res) {
                    const __nv_bfloat162* rr = reinterpret_cast<const __nv_bfloat162*>(&rres[c0 / 8]);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        v[2 * j] += __bfloat162float(rr[j].x);
                        v[2 * j + 1] += __bfloat162float(rr[j].y);
                    }
                }
                if (a.Y) {
                    uint4 w2[2];
                    __nv_bfloat162* wb = reinterpret_cast<__nv_bfloat162*>(w2);
#pragma unroll
                    for (int j = 0; j < 8; ++j) wb[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                    *reinterpret_cast<uint4*>(a.Y + o) = w2[0];
                    *reinterpret_cast<uint4*>(a.Y + o + 8) = w2[1];
                }
                if (a.Yf) {
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(a.Yf + o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
            }
        }
    }
    t5_finish<ST, CS>(bars, tmem, COLS, flags, err);
}

// ---------------------------------------------------------------------------
// Weight gradient dW[tap][co][ci] = sum_p G[p][co] X[p + d off(tap)][ci]
// (X = the layer's input, rectified in shared memory when relu_in; G = the
// gradient of its output).  A block owns one row of taps (dy = blockIdx.x
// - 1, all three dx), a 128-channel tile of one side and an N-channel
// tile of the other (blockIdx.z), and every 64-pixel row segment of one
// split (blockIdx.y): K = pixels, 64 a stage, both operands MN-major (the
// channels are contiguous in memory).  MG: the 128-channel M side is G's
// output channels (N = X's input channels), else it is X's input channels
// (N = G's 16 output channels, the head).  The G tile of a stage is loaded
// once for the three taps; each tap's X tile sits at its own offset, zero
// filled outside the image, and accumulates into its own N columns of
// tensor memory.  The split's sums go to part[split][tap][co][ci] and are
// added in split order afterwards, so every run sums the same way.
//   stage layout: the G tile, then the X tiles of taps dx = -1, 0, 1; a
//   128-channel tile is two 64-channel boxes of 64 rows (pixels) x 128
//   bytes (128-byte swizzle: 8-row groups 1024 bytes apart, the second box
//   8192 bytes on), a 16-channel tile one box of 64 rows x 32 bytes (32-byte
//   swizzle, 8-row groups 256 bytes apart).  A K = 16 step moves 16 rows on.
template <bool MG, int N, int ST>
__global__ void __launch_bounds__(T5_THREADS) ws_wgrad5_kernel(const __grid_constant__ TmaOperands maps,
                                                                const WgradArgs a, int* err)
{
    constexpr uint32_t MSZ = 128 * 64 * 2, NSZ = N * 64 * 2;
    constexpr uint32_t GSZ = MG ? MSZ : NSZ, XSZ = MG ? NSZ : MSZ, SBYTES = GSZ + 3 * XSZ;
    constexpr uint32_t IDESC = t5_idesc(128, N, true, true);
    constexpr uint32_t COLS = t5_cols(3 * N);
    extern __shared__ __align__(16) unsigned char t5_raw[];
    __shared__ __align__(8) T5Bars<ST> bars;
    __shared__ uint32_t tmem_slot;
    __shared__ int flags[3];
    const uint32_t raw = smem_addr(t5_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* tsm = t5_raw + (base - raw);
    const int R = a.R, Cin = a.Cin, Cout = a.Cout, dil = a.dil;
    const int dy = (int)blockIdx.x - 1, split = blockIdx.y;
    const int mtiles = (MG ? Cout : Cin) / 128;
    const int m0 = (blockIdx.z % mtiles) * 128, n0 = (blockIdx.z / mtiles) * N;
    const int g0c = MG ? m0 : n0, x0c = MG ? n0 : m0;  // first channel of the G and X tiles
    const int segs_row = R / 64, segs = a.B * R * segs_row;
    const int sg0 = (int)((long long)split * segs / a.splits), sg1 = (int)((long long)(split + 1) * segs / a.splits);
    const int NS = sg1 - sg0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tmem = t5_start<ST>(bars, &tmem_slot, COLS, flags);

    if (warp == 0) {
        if (lane == 0) {
            int s = 0;
            for (; s < NS; ++s) {
                const int buf = s % ST;
                if (s >= ST && !tc_mbar_wait(smem_addr(&bars.empty[buf]), (uint32_t)(s / ST + 1) & 1u)) {
                    atomicOr(&flags[0], 1);
                    break;
                }
                const int g = sg0 + s, x0 = (g % segs_row) * 64, row = g / segs_row;
                const int y = row % R, b = row / R;
                const uint32_t st = base + buf * SBYTES, bar = smem_addr(&bars.full[buf]);
                t5_expect(bar, SBYTES);
                // G tile (maps.A), box of 64 or 16 channels
                if (GSZ == MSZ) {
                    t5_load4(st, &maps.A, g0c, x0, y, b, bar);
                    t5_load4(st + 8192, &maps.A, g0c + 64, x0, y, b, bar);
                } else {
                    t5_load4(st, &maps.A, g0c, x0, y, b, bar);
                }
                // X tiles of the three taps of this row (maps.B)
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const uint32_t xt = st + GSZ + t * XSZ;
                    const int xx = x0 + (t - 1) * dil, yy = y + dy * dil;
                    if (XSZ == MSZ) {
                        t5_load4(xt, &maps.B, x0c, xx, yy, b, bar);
                        t5_load4(xt + 8192, &maps.B, x0c + 64, xx, yy, b, bar);
                    } else {
                        t5_load4(xt, &maps.B, x0c, xx, yy, b, bar);
                    }
                }
            }
            flags[1] = s;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int s = 0;
            for (; s < NS; ++s) {
                const int buf = s % ST;
                const uint32_t bar = smem_addr(a.relu_in ? &bars.ready[buf] : &bars.full[buf]);
                if (!tc_mbar_wait(bar, (uint32_t)(s / ST) & 1u)) {
                    atomicOr(&flags[0], 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t st = base + buf * SBYTES;
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const uint32_t xt = st + GSZ + t * XSZ;
                    const uint32_t sa = MG ? st : xt;  // the 128-channel side
                    const uint32_t sb = MG ? xt : st;  // the N side
#pragma unroll
                    for (int k16 = 0; k16 < 4; ++k16) {
                        const uint64_t ad = t5_desc(sa + k16 * 2048, 8192, 1024, T5_SW128);
                        const uint64_t bd = N == 128 ? t5_desc(sb + k16 * 2048, 8192, 1024, T5_SW128)
                                                     : t5_desc(sb + k16 * 512, 16, 256, T5_SW32);
                        t5_mma(tmem + t * N, ad, bd, IDESC, (s | k16) != 0 ? 1u : 0u);
                    }
                }
                t5_commit(smem_addr(&bars.empty[buf]));
            }
            if (!a.relu_in) flags[2] = s;
            t5_commit(smem_addr(&bars.done));
        }
        __syncwarp();
    } else {
        if (a.relu_in) {
            int s = 0;
            for (; s < NS; ++s) {
                const int buf = s % ST;
                if (!t5_warp_wait(smem_addr(&bars.full[buf]), (uint32_t)(s / ST) & 1u, lane)) {
                    if (lane == 0) atomicOr(&flags[0], 1);
                    break;
                }
                t5_rectify(tsm + buf * SBYTES + GSZ, 3 * XSZ, tid - 64, T5_THREADS - 64);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncwarp();
                if (lane == 0) t5_arrive(smem_addr(&bars.ready[buf]));
            }
            if (warp == 2 && lane == 0) flags[2] = s;
        }
        const bool fin = t5_warp_wait(smem_addr(&bars.done), 0, lane);
        if (!fin && lane == 0) atomicOr(&flags[0], 1);
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (fin && !*(volatile int*)&flags[0]) {
            const int q = warp & 3;
            const int m = m0 + q * 32 + lane;  // this lane's channel on the 128-channel side
#pragma unroll 1
            for (int t = 0; t < 3; ++t) {
                const int tap = (dy + 1) * 3 + t;
                float* out = a.part + ((size_t)split * 9 + tap) * Cout * Cin;
#pragma unroll 1
                for (int c0 = 0; c0 < N; c0 += 16) {
                    uint32_t r[16];
                    t5_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * N + c0), r);
                    if (MG) {  // row co = m, columns ci = n0 + c0 ..
                        float* d = out + (size_t)m * Cin + n0 + c0;
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4*>(d + j) = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                                                            __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                    } else {  // ci = m, co = n0 + c0 + j: a warp writes 32 consecutive ci
#pragma unroll
                        for (int j = 0; j < 16; ++j) out[(size_t)(n0 + c0 + j) * Cin + m] = __uint_as_float(r[j]);
                    }
                }
            }
        }
    }
    t5_finish<ST>(bars, tmem, COLS, flags, err);
}
