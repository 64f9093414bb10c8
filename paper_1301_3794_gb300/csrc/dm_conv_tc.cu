// Tensor-core (tcgen05) convolutions of the learned smoother.
//
// A zero-padded 3x3x3 convolution on the padded node grid is an implicit GEMM
// over the flattened node index p = off0 + i + sx (j + sy k):
//     out[p, n] = sum_t sum_k Weff[t][k][n] in[p + d_t, k],
//     d_t = (c - 1) + (b - 1) sx + (a - 1) sx sy  for tap t = (a b c) (a along k).
// One tile is 128 consecutive nodes (the MMA's M = 128 rows), N = 16 output
// channels (fewer are zero-padded), and each MMA step takes K = 16 input
// values: one tap of 16 channels, or two taps of 8 channels.
//
// Activations use the channel-blocked layout of ActLayout: channel c of node p
// at ((c / 8) npe + marg + p) * 8 + c % 8 (BF16).  Eight channels of one node
// are one 16-byte row, consecutive nodes are consecutive rows, so the rows a
// tap needs for a tile form one contiguous window of global memory.  For each
// (a, b) and channel block the kernel copies the 130-node window p0 + d_ab - 1
// .. p0 + d_ab + 128 into shared memory with one cp.async.bulk (the margins of
// the layout keep every window inside the buffer); the three taps c = 0, 1, 2
// of that window are the same rows shifted by 16 bytes, i.e. the same window
// with the descriptor's start address moved by one row.
//
// Operands are in the canonical K-major layout without swizzle: core matrices
// of 8 rows x 16 bytes with rows 16 bytes apart; SBO = 128 bytes between
// consecutive 8-row groups (M or N), LBO = the distance between the two
// 16-byte K halves (the second channel block's window, or the second tap's
// rows).  The accumulator (128 lanes x 16 FP32 columns) lives in tensor memory;
// each of the 4 warps reads its 32 lanes back with tcgen05.ld for the epilogue.
//
// Every wait on an mbarrier gives up after about a second: the kernel then
// records an error code, stops issuing work and releases its tensor memory.
#include "dm_common.cuh"
#include "dm_learned.cuh"

#include <cstdint>

namespace dm {

namespace {

constexpr int kTileM = 128;                 // nodes per tile (MMA M)
constexpr int kWin = kTileM + 2;            // window rows: one extra node on each side
constexpr int kWinBytes = kWin * 16;        // 2080
constexpr int kStepBytes = 2 * 16 * 16 * 2; // one step's B tiles (N = 16, K = 16, BF16): high part, low part
constexpr uint32_t kTmemCols = 32;          // smallest allocation; columns 0..15 used
constexpr unsigned long long kWaitNs = 1000000000ull;   // one second

// instruction descriptor of tcgen05.mma kind::f16: BF16 A and B (K-major),
// FP32 accumulator, M = 128, N = 16
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// true once the phase of parity `parity` completed; false after kWaitNs
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// warp-wide
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
// shared-memory matrix descriptor: no swizzle, version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_bf16_id(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// this thread's lane (row), 16 consecutive FP32 columns from `taddr`
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// node (i, j, k) of padded index p is a grid node (0 <= i <= nx, ...)
__device__ __forceinline__ bool grid_node(const Grid3& g, int p) {
    const int kk = p / g.sxy, rem = p - kk * g.sxy;
    const int jj = rem / g.sx, ii = rem - jj * g.sx;
    return ii >= 1 && ii <= g.nx + 1 && jj >= 1 && jj <= g.ny + 1 && kk >= 1 && kk <= g.nz + 1;
}

// B tiles of every MMA step, BF16 canonical K-major (N = 16 rows, K = 16):
// element (n, k) of step s at s * 512 + h * 256 + (k / 8) * 128 + (n / 8) * 64 +
// (n % 8) * 8 + k % 8, where h = 0 holds the weight rounded to BF16 and h = 1
// the BF16 rounding of what is left (w - hi): the two MMAs of a step then
// multiply by the weight to about 16 significant bits, which the residual
// objective needs (its gradient passes the output through K twice, and BF16
// weights alone would leave a 1.5% gradient error).
// CB = 2: step s is tap s with k = input channel 0..15.  CB = 1: step s < 13
// holds taps 2s (k < 8) and 2s + 1 (k >= 8, channel k - 8); step 13 holds tap
// 26 in its upper half and zero weights in its lower half (whose rows the
// kernel points at finite data below tap 26's, so the K stride stays positive).
// Weff[t][k][n] = W[t][k][n] (forward, W: [27][cin][cout]), or for the adjoint
// of a forward conv with weights W: [27][cout'][cin'], W[26 - t][n][k].
__global__ void k_pack_wtiles(const float* __restrict__ W, int wcin, int wcout, int cin, int cout, int cb, int flip,
                              __nv_bfloat16* __restrict__ out) {
    const int nsteps = cb == 2 ? 27 : 14;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nsteps * 256; e += gridDim.x * blockDim.x) {
        const int s = e / 256, r = e % 256;
        __nv_bfloat16* const o = out + s * 512 + r;
        const int kh = r / 128, r2 = r % 128, ng = r2 / 64, r3 = r2 % 64, n = ng * 8 + r3 / 8, kl = r3 % 8;
        const int kin = kh * 8 + kl;
        int t, ch;
        if (cb == 2) {
            t = s;
            ch = kin;
        } else {
            t = s < 13 ? 2 * s + kh : (kh ? 26 : 27);
            ch = kl;
        }
        float v = 0.f;
        if (t < 27 && ch < cin && n < cout)
            v = flip ? W[((size_t)(26 - t) * wcin + n) * wcout + ch] : W[((size_t)t * wcin + ch) * wcout + n];
        const __nv_bfloat16 hi = __float2bfloat16(v);
        o[0] = hi;
        o[256] = __float2bfloat16(v - __bfloat162float(hi));
    }
}

enum ConvEpi { EPI_RELU_BF16 = 0, EPI_MASK_BF16 = 1, EPI_F32_3 = 2 };

// One CTA of 128 threads (4 warps) takes tiles t = tile0 + blockIdx.x, +gridDim.x, ...
template <int CB, int EPI>
__global__ void __launch_bounds__(128) k_conv_tc(Grid3 g, ActLayout L, const __nv_bfloat16* __restrict__ in,
                                                 const __nv_bfloat16* __restrict__ wtiles,
                                                 const __nv_bfloat16* __restrict__ mask,
                                                 __nv_bfloat16* __restrict__ out, float* __restrict__ outY, int tile0,
                                                 int ntiles, int* __restrict__ err) {
    constexpr int kSteps = CB == 2 ? 27 : 14;
    constexpr int kChunks = 9 * CB;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* s_w = smem;                                   // kSteps B tiles
    unsigned char* s_win = smem + kSteps * kStepBytes;           // kChunks windows (+ slack)
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights: global BF16 tiles -> shared (generic proxy), made visible to the tensor cores below
    {
        const uint4* src = reinterpret_cast<const uint4*>(wtiles);
        uint4* dst = reinterpret_cast<uint4*>(s_w);
        for (int e = tid; e < kSteps * kStepBytes / 16; e += 128) dst[e] = src[e];
    }
    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        s_abort = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&s_tmem, kTmemCols);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t w_base = smem_u32(s_w), win_base = smem_u32(s_win);
    uint32_t phase = 0;

    for (int t = tile0 + blockIdx.x; t < tile0 + ntiles; t += gridDim.x) {
        const int p0 = t * kTileM;
        if (tid == 0) {
            mbar_expect_tx(&bar_load, kChunks * kWinBytes);
#pragma unroll 1
            for (int ab = 0; ab < 9; ++ab) {
                const int a = ab / 3, b = ab % 3;
                const int q = p0 + (b - 1) * g.sx + (a - 1) * g.sxy - 1;
#pragma unroll
                for (int cb = 0; cb < CB; ++cb)
                    bulk_g2s(s_win + (ab * CB + cb) * kWinBytes, in + L.at(cb, q), kWinBytes, &bar_load);
            }
        }
        if (!mbar_wait(&bar_load, phase)) {
            atomicExch(err, 1);
            s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        if (tid == 0) {
            tc_fence_after();
#pragma unroll 1
            for (int s = 0; s < kSteps; ++s) {
                uint32_t a0, lbo;
                if (CB == 2) {
                    const int ab = s / 3, c = s % 3;
                    a0 = win_base + ab * CB * kWinBytes + c * 16;
                    lbo = kWinBytes;   // second channel block's window
                } else if (s < 13) {
                    const int t1 = 2 * s, t2 = t1 + 1;
                    a0 = win_base + (t1 / 3) * kWinBytes + (t1 % 3) * 16;
                    lbo = win_base + (t2 / 3) * kWinBytes + (t2 % 3) * 16 - a0;
                } else {
                    // lower half: zero weights on tap 0's rows (finite data); upper half: tap 26
                    a0 = win_base;
                    lbo = 8 * kWinBytes + 2 * 16;
                }
                const uint64_t ad = sdesc(a0, lbo, 128);
                mma_bf16(tmem, ad, sdesc(w_base + s * kStepBytes, 256, 128), s > 0 ? 1u : 0u);
                mma_bf16(tmem, ad, sdesc(w_base + s * kStepBytes + 512, 256, 128), 1u);
            }
            mma_commit(&bar_mma);
        }
        if (!mbar_wait(&bar_mma, phase)) {
            atomicExch(err, 2);
            s_abort = 1;
        }
        tc_fence_after();
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
        const int p = p0 + warp * 32 + lane;
        if (p < L.np) {
            const bool ok = grid_node(g, p) && !s_abort;
            if (EPI == EPI_F32_3) {
#pragma unroll
                for (int c = 0; c < 3; ++c) outY[(size_t)p * 3 + c] = ok ? v[c] : 0.f;
            } else {
#pragma unroll
                for (int cb = 0; cb < 2; ++cb) {
                    float m[8];
                    if (EPI == EPI_MASK_BF16) {
                        const uint4 mv = *reinterpret_cast<const uint4*>(mask + L.at(cb, p));
                        const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mv);
#pragma unroll
                        for (int c = 0; c < 8; ++c) m[c] = __bfloat162float(mb[c]) > 0.f ? 1.f : 0.f;
                    }
                    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float x = v[cb * 8 + c];
                        if (EPI == EPI_RELU_BF16) x = fmaxf(x, 0.f);
                        else x *= m[c];
                        o[c] = __float2bfloat16(ok ? x : 0.f);
                    }
                    *reinterpret_cast<uint4*>(out + L.at(cb, p)) = *reinterpret_cast<const uint4*>(o);
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        if (s_abort) break;
        phase ^= 1u;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// shared bytes of a conv kernel: B tiles, windows, and slack so that a
// descriptor with its two strides exchanged still stays inside the allocation
template <int CB>
constexpr size_t conv_smem() {
    return (size_t)(CB == 2 ? 27 : 14) * kStepBytes + (size_t)9 * CB * kWinBytes + 16 * kWinBytes;
}

template <int CB, int EPI>
void conv_tc_launch(const Grid3& g, const ActLayout& L, const __nv_bfloat16* in, const __nv_bfloat16* wt,
                    const __nv_bfloat16* mask, __nv_bfloat16* out, float* outY, int* err, cudaStream_t s) {
    const size_t sm = conv_smem<CB>();
    static bool attr = false;   // set once per process (all devices share the kernel's attribute)
    if (!attr) {
        DM_CUDA(cudaFuncSetAttribute(k_conv_tc<CB, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = true;
    }
    const int first = g.off0 / kTileM;
    const int last = g.idx(g.nx, g.ny, g.nz) / kTileM;
    const int ntiles = last - first + 1;
    int per_sm = 0;
    DM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_tc<CB, EPI>, 128, sm));
    int dev = 0, sms = 0;
    DM_CUDA(cudaGetDevice(&dev));
    DM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::max(1, std::min(ntiles, sms * std::max(per_sm, 1)));
    // bytes: every input block's nodes once, the output once
    const double bytes = (double)L.np * (16.0 * CB + (EPI == EPI_F32_3 ? 12.0 : 32.0 + (EPI == EPI_MASK_BF16 ? 32.0 : 0.0)));
    launch_b(EPI == EPI_F32_3 ? "conv_tc_out" : (EPI == EPI_MASK_BF16 ? "conv_tc_adjoint" : "conv_tc_relu"), bytes,
             k_conv_tc<CB, EPI>, grid, 128, sm, s, g, L, in, wt, mask, out, outY, first, ntiles, err);
}

// ---- weight gradient --------------------------------------------------------
//
// dW[t][ci][co] = sum_p in[p + d_t, ci] dy[p, co] is a GEMM whose reduction
// runs over nodes: D[m][n] = sum_k A[m][k] B[n][k] with m = (tap, ci), n = co,
// k = node.  Both operands are MN-major (the 8 channels of one node are
// contiguous): core matrices of 8 nodes (K) x 16 bytes (8 channels), nodes 16
// bytes apart; LBO = 128 bytes between consecutive 8-node groups (K), SBO =
// 2048 bytes between consecutive 8-channel groups (M or N), which are separate
// 128-node windows: tap t's window of channel block cb for an M tile of 16 / CB
// taps.  An M tile holds 16 groups (8 taps of 16 channels, or 16 taps of 8);
// 27 taps take 4 or 2 M tiles, each accumulating in its own 16 TMEM columns
// over every node tile the CTA visits.  Rows of taps past 26 and columns past
// cout hold whatever the slots contain and are never read out.
constexpr int kDwSlot = kTileM * 16;     // one 128-node window of 8 channels
constexpr uint32_t kIdescMN = kIdesc | (1u << 15) | (1u << 16);
constexpr int kDwCtasPerSm = 4;

template <int CB>
__global__ void __launch_bounds__(128) k_conv_dw_tc(Grid3 g, ActLayout L, const __nv_bfloat16* __restrict__ in,
                                                    int cb_out, const __nv_bfloat16* __restrict__ dy, int tile0,
                                                    int ntiles, float* __restrict__ part, int* __restrict__ err) {
    constexpr int kTapsPerM = 16 / CB;
    constexpr int kMTiles = (27 + kTapsPerM - 1) / kTapsPerM;
    constexpr uint32_t kCols = kMTiles * 16 <= 32 ? 32 : 64;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* s_a = smem;                    // 16 slots
    unsigned char* s_b = smem + 16 * kDwSlot;     // 2 slots (channel blocks of dy)
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        s_abort = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&s_tmem, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t a_base = smem_u32(s_a), b_base = smem_u32(s_b);
    uint32_t phase = 0;
    bool first = true;
    for (int t = tile0 + blockIdx.x; t < tile0 + ntiles && !s_abort; t += gridDim.x) {
        const int p0 = t * kTileM;
        for (int mt = 0; mt < kMTiles; ++mt) {
            if (tid == 0) {
                const int nt = min(kTapsPerM, 27 - mt * kTapsPerM);
                mbar_expect_tx(&bar_load, (uint32_t)(nt * CB + (mt == 0 ? cb_out : 0)) * kDwSlot);
#pragma unroll 1
                for (int tl = 0; tl < nt; ++tl) {
                    const int tap = mt * kTapsPerM + tl;
                    const int a = tap / 9, b = (tap / 3) % 3, c = tap % 3;
                    const int q = p0 + (c - 1) + (b - 1) * g.sx + (a - 1) * g.sxy;
                    for (int cb = 0; cb < CB; ++cb)
                        bulk_g2s(s_a + (tl * CB + cb) * kDwSlot, in + L.at(cb, q), kDwSlot, &bar_load);
                }
                if (mt == 0)
                    for (int cb = 0; cb < cb_out; ++cb) bulk_g2s(s_b + cb * kDwSlot, dy + L.at(cb, p0), kDwSlot, &bar_load);
            }
            if (!mbar_wait(&bar_load, phase)) {
                atomicExch(err, 3);
                s_abort = 1;
            }
            __syncthreads();
            if (s_abort) break;
            if (tid == 0) {
                tc_fence_after();
#pragma unroll 1
                for (int kk = 0; kk < kTileM / 16; ++kk)
                    mma_bf16_id(tmem + mt * 16, sdesc(a_base + kk * 256, 128, kDwSlot),
                                sdesc(b_base + kk * 256, 128, kDwSlot), kIdescMN, (first && kk == 0) ? 0u : 1u);
                mma_commit(&bar_mma);
            }
            if (!mbar_wait(&bar_mma, phase)) {
                atomicExch(err, 4);
                s_abort = 1;
            }
            phase ^= 1u;
            __syncthreads();
            if (s_abort) break;
        }
        first = false;
    }
    // read out this CTA's sums: lane = row m of each M tile, 16 columns per M tile
    tc_fence_after();
    float* out = part + (size_t)blockIdx.x * 27 * 256;
    const int m = warp * 32 + lane, grp = m / 8, tl = grp / CB, cb = grp % CB, ci = cb * 8 + (m % 8);
    for (int mt = 0; mt < kMTiles; ++mt) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + mt * 16, v);
        const int tap = mt * kTapsPerM + tl;
        if (tap < 27 && ci < 16)
#pragma unroll
            for (int n = 0; n < 16; ++n) out[((size_t)tap * 16 + ci) * 16 + n] = (first || s_abort) ? 0.f : v[n];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// dW[t][ci][co] = sum over CTAs (in CTA order) of part[cta][t][ci][co]
__global__ void k_dw_sum(const float* __restrict__ part, int nparts, int cin, int cout, float* __restrict__ dW) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 27 * cin * cout) return;
    const int t = e / (cin * cout), r = e % (cin * cout), ci = r / cout, co = r % cout;
    float s = 0.f;
    for (int b = 0; b < nparts; ++b) s += part[((size_t)b * 27 + t) * 256 + ci * 16 + co];
    dW[e] = s;
}

}  // namespace

int conv_dw_tc_parts() {
    int dev = 0, sms = 0;
    DM_CUDA(cudaGetDevice(&dev));
    DM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms * kDwCtasPerSm;
}

void conv_dw_tc(const Grid3& g, const ActLayout& L, int cb_in, int cin, const __nv_bfloat16* in, int cb_out, int cout,
                const __nv_bfloat16* dy, float* part, float* dW, int* err, cudaStream_t s) {
    DM_REQUIRE((cb_in == 1 || cb_in == 2) && cin <= 8 * cb_in && cout <= 8 * cb_out && cb_out >= 1 && cb_out <= 2,
               DM_ERR_INVALID_ARG, "conv_dw_tc: channel counts");
    const size_t sm = 18 * (size_t)kDwSlot + 8192;   // 16 A slots, 2 B slots, slack
    static bool attr1 = false, attr2 = false;
    const int first = g.off0 / kTileM, last = g.idx(g.nx, g.ny, g.nz) / kTileM, ntiles = last - first + 1;
    const int nparts = std::min(conv_dw_tc_parts(), ntiles);
    // bytes: every node of the input blocks 27 times from L2 is not DRAM traffic; count the input and dy once
    const double bytes = (double)L.np * 16.0 * (cb_in + cb_out);
    if (cb_in == 2) {
        if (!attr2) {
            DM_CUDA(cudaFuncSetAttribute(k_conv_dw_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            attr2 = true;
        }
        launch_b("conv_tc_dw", bytes, k_conv_dw_tc<2>, nparts, 128, sm, s, g, L, in, cb_out, dy, first, ntiles, part,
                 err);
    } else {
        if (!attr1) {
            DM_CUDA(cudaFuncSetAttribute(k_conv_dw_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            attr1 = true;
        }
        launch_b("conv_tc_dw", bytes, k_conv_dw_tc<1>, nparts, 128, sm, s, g, L, in, cb_out, dy, first, ntiles, part,
                 err);
    }
    const int n = 27 * cin * cout;
    launch("conv_tc_dw_sum", k_dw_sum, (n + 127) / 128, 128, 0, s, (const float*)part, nparts, cin, cout, dW);
}

ActLayout act_layout(const Grid3& g) {
    ActLayout L;
    L.np = g.np;
    // windows reach sxy + sx + 1 nodes below a tile and as far above its end;
    // the last tile may also run up to 127 nodes past np
    L.marg = ((g.sxy + g.sx + 2 + 7) / 8) * 8 + kTileM;
    L.npe = g.np + 2 * L.marg;
    return L;
}

int conv_wtile_steps(int cb) { return cb == 2 ? 27 : 14; }

void conv_pack_weights(const float* W, int wcin, int wcout, int cin, int cout, int cb, int flip, __nv_bfloat16* out,
                       cudaStream_t s) {
    launch("conv_tc_pack", k_pack_wtiles, 32, 256, 0, s, W, wcin, wcout, cin, cout, cb, flip, out);
}

void conv_tc(const Grid3& g, const ActLayout& L, int cb, int epi, const __nv_bfloat16* in, const __nv_bfloat16* wt,
             const __nv_bfloat16* mask, __nv_bfloat16* out, float* outY, int* err, cudaStream_t s) {
    if (cb == 1 && epi == EPI_RELU_BF16) conv_tc_launch<1, EPI_RELU_BF16>(g, L, in, wt, mask, out, outY, err, s);
    else if (cb == 1 && epi == EPI_MASK_BF16) conv_tc_launch<1, EPI_MASK_BF16>(g, L, in, wt, mask, out, outY, err, s);
    else if (cb == 2 && epi == EPI_RELU_BF16) conv_tc_launch<2, EPI_RELU_BF16>(g, L, in, wt, mask, out, outY, err, s);
    else if (cb == 2 && epi == EPI_MASK_BF16) conv_tc_launch<2, EPI_MASK_BF16>(g, L, in, wt, mask, out, outY, err, s);
    else if (cb == 2 && epi == EPI_F32_3) conv_tc_launch<2, EPI_F32_3>(g, L, in, wt, mask, out, outY, err, s);
    else throw Error(DM_ERR_INVALID_ARG, "conv_tc: unsupported channel blocks / epilogue");
}

}  // namespace dm
