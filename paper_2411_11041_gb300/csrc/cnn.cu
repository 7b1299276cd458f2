// Warm-start network on the GPU: BF16 tensor-core convolutions with FP32
// accumulation (forward, data gradient, weight gradient), loss, Adam, and the
// feature / target / unpacking kernels.  See include/adr.h (adr_cnn_*).
//
// Network (the same definition as the FP64 reference): a 256 x 256 node grid
// is read as 64 x 64 cells of 4 x 4 nodes, every problem scaled by
// s = max |u0| of its first initial state u0; features NHWC, 40 channels (f
// and u0 / s at the 16 nodes of the cell; cell means of beta1, beta2, mu and
// sigma codes, cell mean of the mask, 3 zeros); eight 3 x 3 convolutions with
// zero padding, channels 40 64 64 128 128 128 64 64 8, bias, ReLU after all
// but the last; output channel 0 = the cell mean of (u - u0) / s, channels
// 1..7 unused; initial state u0 + s * (bilinear interpolation of channel 0).
// Parameters packed as W_0, b_0, W_1, b_1, ...; W_l[(tap * Cin + ci) * Cout + co].
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "adr_internal.cuh"

namespace {

constexpr int kLayers = 8;
constexpr int kCh[kLayers + 1] = {40, 64, 64, 128, 128, 128, 64, 64, 8};
constexpr int kDil[kLayers] = {1, 2, 4, 8, 16, 32, 1, 1};
constexpr int kHW = 64;   // cells per side
constexpr int kSub = 4;   // nodes per cell side
constexpr int kN = kHW * kSub;
constexpr int kCin = 40, kCout = 8;

long param_offset(int l, bool bias)
{
    long off = 0;
    for (int k = 0; k < l; ++k) off += 9L * kCh[k] * kCh[k + 1] + kCh[k + 1];
    return bias ? off + 9L * kCh[l] * kCh[l + 1] : off;
}

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool ok)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(ok ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned (&r)[2], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ------------------------------------------------------ convolution kernels

struct ConvArgs {
    int B, H, W, Cin, Cout, dil;
    const bf16* x;      // [B][H][W][Cin]
    const bf16* w;      // [9 Cin][Cout]
    const float* bias;  // [Cout] or null
    bf16* y;            // [B][H][W][Cout] or null
    float* y32;         // [B][H][W][Cout] FP32 output or null
    int relu;
    long long spin;     // tensor-core kernels: bound of their mbarrier waits in polls
                        // (0: the default bound)
};

// implicit GEMM: M = pixels, N = Cout, K = 9 Cin (tap-major); a block computes
// 128 pixels x BN channels with 8 warps; double-buffered cp.async tiles.
template <int BN>
__global__ void __launch_bounds__(256) k_conv_fwd(ConvArgs a)
{
    constexpr int BM = 128, BK = 32, AS = BK + 8, BSTR = BN + 8;
    constexpr int WN = BN >= 64 ? 2 : 1, WM = 8 / WN, TM = BM / WM, TN = BN / WN;
    constexpr int MI = TM / 16, NI = TN / 8;
    __shared__ __align__(16) bf16 As[2][BM][AS];
    __shared__ __align__(16) bf16 Bs[2][BK][BSTR];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp / WN, wn = warp % WN;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int HW = a.H * a.W;
    const long long M = (long long)a.B * HW;
    const int K = 9 * a.Cin;
    float acc[MI][NI][4];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;

    auto load = [&](int st, int k0) {
        for (int v = tid; v < BM * (BK / 8); v += 256) {
            int row = v / (BK / 8), kg = v % (BK / 8);
            long long p = m0 + row;
            int k = k0 + kg * 8;
            const bf16* src = a.x;
            bool ok = false;
            if (p < M && k < K) {
                int tap = k / a.Cin, ci = k - tap * a.Cin;
                int b = (int)(p / HW), rem = (int)(p - (long long)b * HW);
                int r = rem / a.W, c = rem - r * a.W;
                int rr = r + (tap / 3 - 1) * a.dil, cc = c + (tap % 3 - 1) * a.dil;
                if (rr >= 0 && rr < a.H && cc >= 0 && cc < a.W) {
                    src = a.x + (((long long)b * a.H + rr) * a.W + cc) * a.Cin + ci;
                    ok = true;
                }
            }
            cp_async16(&As[st][row][kg * 8], src, ok);
        }
        for (int v = tid; v < BK * (BN / 8); v += 256) {
            int row = v / (BN / 8), ng = v % (BN / 8);
            int k = k0 + row, n = n0 + ng * 8;
            bool ok = k < K && n < a.Cout;
            cp_async16(&Bs[st][row][ng * 8], ok ? a.w + (long long)k * a.Cout + n : a.w, ok);
        }
        cp_async_commit();
    };
    const int nk = (K + BK - 1) / BK;
    load(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt + 1 < nk) {
            load(st ^ 1, (kt + 1) * BK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[MI][4], bfr[NI][2];
#pragma unroll
            for (int i = 0; i < MI; ++i)
                ldsm_x4(af[i], &As[st][wm * TM + i * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
            for (int j = 0; j < NI; ++j) ldsm_x2_t(bfr[j], &Bs[st][kk + (lane & 15)][wn * TN + j * 8]);
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < NI; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j) {
            int n = n0 + wn * TN + j * 8 + 2 * t;
            if (n >= a.Cout) continue;
            float b0 = a.bias ? a.bias[n] : 0.f, b1 = a.bias ? a.bias[n + 1] : 0.f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                long long p = m0 + wm * TM + i * 16 + g + h * 8;
                if (p >= M) continue;
                float v0 = acc[i][j][2 * h] + b0, v1 = acc[i][j][2 * h + 1] + b1;
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (a.y)
                    *reinterpret_cast<__nv_bfloat162*>(a.y + p * a.Cout + n) = __floats2bfloat162_rn(v0, v1);
                if (a.y32) {
                    a.y32[p * a.Cout + n] = v0;
                    a.y32[p * a.Cout + n + 1] = v1;
                }
            }
        }
}

// ------------------------------------------------ tensor-core convolution
// The same implicit GEMM on the 5th-generation tensor cores: tcgen05.mma
// (kind::f16, BF16 operands, FP32 accumulator in tensor memory), one CTA of
// 128 threads per 128 output pixels and all N = Cout output channels.  A
// (im2col rows) and B (weights, K-major) are staged by cp.async into shared
// memory in the 128-byte-swizzled K-major layout, two stages deep; one thread
// issues the MMAs of a stage and commits them to that stage's mbarrier, which
// frees the stage for the copies two steps later.  The epilogue reads the
// accumulator rows back with tcgen05.ld (thread t <-> row t), adds the bias,
// applies the ReLU and stores BF16.  Every mbarrier wait is bounded; when a
// wait gives up the kernel sets *err, lets the MMAs it issued finish, skips
// the epilogue and frees its tensor memory.  The decision to give up is the
// block's (every thread agrees), so the barriers and the warp-collective
// tensor-memory loads are never reached by part of a block.

constexpr long long kWaitLimit = 1LL << 22;  // default bound: blocking polls (about a second)

__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the leading offset is not used by this layout)
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N
__device__ __forceinline__ uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Wait for the phase of parity `parity` of an mbarrier.  spin <= 0: up to
// kWaitLimit blocking polls (try_wait); spin > 0: up to spin non-blocking
// polls (test_wait), a bound a caller sets to exercise the give-up path.
// Gives up by setting *err and returning false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, long long spin = 0)
{
    if (spin > 0) {
        for (long long it = 0; it < spin; ++it) {
            uint32_t ok;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(bar), "r"(parity)
                : "memory");
            if (ok) return true;
        }
    } else {
        for (long long it = 0; it < kWaitLimit; ++it) {
            uint32_t ok;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(bar), "r"(parity)
                : "memory");
            if (ok) return true;
        }
    }
    atomicExch(err, 1);
    return false;
}

template <int N>
__global__ void __launch_bounds__(128) k_conv_tc(ConvArgs a, int* err)
{
    constexpr int BK = 64, A_BYTES = 128 * 128, B_BYTES = N * 128, STAGE = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int HW = a.H * a.W;
    const long long M = (long long)a.B * HW, m0 = (long long)blockIdx.x * 128;
    const int K = 9 * a.Cin;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    // this thread stages the 16-byte K chunk c of the rows r = tid/8 + 16 i
    const int c = tid & 7, r0 = tid >> 3;
    int pb[8], py[8], px[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        long long m = m0 + r0 + 16 * i;
        if (m < M) {
            int b = (int)(m / HW), rem = (int)(m - (long long)b * HW);
            pb[i] = b;
            py[i] = rem / a.W;
            px[i] = rem - py[i] * a.W;
        } else {
            pb[i] = -1;
            py[i] = px[i] = 0;
        }
    }
    const int nk = (K + BK - 1) / BK;
    bool ok = true;
    int issued = 0;  // steps whose MMAs were issued and committed
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (kt >= 2) {
            // the stage's previous MMAs (step kt - 2) must be done; the block decides together
            const bool w = mbar_wait(smem_u32(&mbar[st]), ((kt - 2) >> 1) & 1, err, a.spin);
            ok = __syncthreads_and(w ? 1 : 0) != 0;
            if (!ok) break;
        }
        const uint32_t sa = sbase + st * STAGE, sb = sa + A_BYTES;
        const int k = kt * BK + c * 8;
        const bool kin = k < K;
        const int tap = kin ? k / a.Cin : 0, ci = k - tap * a.Cin;
        const int dy = (tap / 3 - 1) * a.dil, dx = (tap % 3 - 1) * a.dil;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = r0 + 16 * i;
            const int yy = py[i] + dy, xx = px[i] + dx;
            const bool in = kin && pb[i] >= 0 && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const bf16* src = in ? a.x + (((long long)pb[i] * a.H + yy) * a.W + xx) * a.Cin + ci : a.x;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa + sw128(r, c)), "l"(src),
                         "r"(in ? 16 : 0));
        }
#pragma unroll
        for (int i = 0; i < N / 16; ++i) {
            const int r = r0 + 16 * i;  // output channel
            const bf16* src = kin ? a.w + (long long)r * K + k : a.w;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sb + sw128(r, c)), "l"(src),
                         "r"(kin ? 16 : 0));
        }
        asm volatile("cp.async.commit_group;\n");
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t idesc = umma_idesc(128, N);
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
                const uint64_t ad = umma_sdesc(sa + ks * 32), bd = umma_sdesc(sb + ks * 32);
                const uint32_t acc = (kt > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&mbar[st])));
        }
        issued = kt + 1;
        __syncthreads();
    }
    // the last commit arrives once every MMA the thread issued is done
    if (issued >= 1) {
        const uint32_t bar = smem_u32(&mbar[(issued - 1) & 1]), par = ((issued - 1) >> 1) & 1;
        bool w = ok && mbar_wait(bar, par, err, a.spin);
        if (!w) mbar_wait(bar, par, err);  // gave up: let the MMAs finish before the memory is freed
        ok = __syncthreads_and((ok && w) ? 1 : 0) != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (ok) {
        const long long m = m0 + tid;  // accumulator row = tensor-memory lane
        const uint32_t lane = (uint32_t)(warp * 32) << 16;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(tmem + lane + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (m < M) {
                uint32_t packed[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float f0 = __uint_as_float(v[2 * j]), f1 = __uint_as_float(v[2 * j + 1]);
                    if (a.bias) {
                        f0 += a.bias[c0 + 2 * j];
                        f1 += a.bias[c0 + 2 * j + 1];
                    }
                    if (a.relu) {
                        f0 = fmaxf(f0, 0.f);
                        f1 = fmaxf(f1, 0.f);
                    }
                    __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
                    packed[j] = *reinterpret_cast<uint32_t*>(&h);
                }
                uint4* dst = reinterpret_cast<uint4*>(a.y + m * N + c0);
                dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(N));
}

// ------------------------------------------------ TMA-fed tensor-core convolution
// For inputs of 64 or 128 channels: a CTA computes the output pixels of an
// 8 MT x 16 window of one image for all N output channels.  The K loop runs over
// (tap, 64-channel block); for each, one TMA load brings the input window
// shifted by the tap's offset (the image border comes as TMA's zero fill) and
// one brings the 64 x N weight tile, both with the 128-byte swizzle, which is
// the K-major layout the MMA descriptors expect (row = pixel y * 16 + x).
// Thread 0 (the producer) keeps up to S stages in flight on "full" mbarriers
// (transaction bytes); thread 32 (the MMA issuer, another warp) issues a
// stage's MMAs as soon as it lands, and their commit to the stage's "empty"
// mbarrier frees it for the producer.  The MMAs of consecutive stages queue
// back to back.  Every wait is bounded; on a timeout the kernel sets *err,
// waits (bounded) for the loads it issued that no MMA consumed, skips the
// epilogue and frees its tensor memory.
// MT windows of 8 x 16 pixels stacked (an 8 MT x 16 window, one TMA load),
// each with its own accumulator (tensor-memory columns [t N, t N + N)),
// sharing every weight tile.  Measured on the 128-problem forward pass with
// one thread loading and issuing: one window 1.42 ms (3 or 4 stages), two
// windows with 2 stages (two CTAs per SM) 1.11 ms, two with 3 stages 1.48 ms,
// four windows 1.22 ms; with the producer and the MMA issuer apart, two
// windows 1.06 ms with 2 stages and 1.29 ms with 3 (one CTA per SM).
constexpr int kTmaMT = 2;
template <int N>
struct TmaConv {
    static constexpr int MT = kTmaMT;
    static constexpr int S = MT == 1 ? (N == 128 ? 3 : 4) : 2;
    static constexpr int A_BYTES = MT * 128 * 128, B_BYTES = N * 128, STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = S * STAGE + 1024;
    static constexpr int THREADS = 128 * MT;
};

template <int N>
__global__ void __launch_bounds__(TmaConv<N>::THREADS) k_conv_tma(const __grid_constant__ CUtensorMap ta,
                                                                  const __grid_constant__ CUtensorMap tw,
                                                                  ConvArgs a, int* err)
{
    using C = TmaConv<N>;
    constexpr int S = C::S, A_BYTES = C::A_BYTES, STAGE = C::STAGE, MT = C::MT, WH = 8 * MT;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    __shared__ uint64_t full[S], empty[S];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tiles_x = a.W / 16, per_img = tiles_x * (a.H / WH);
    const int b = blockIdx.x / per_img, t = blockIdx.x - b * per_img;
    const int y0 = (t / tiles_x) * WH, x0 = (t - (t / tiles_x) * tiles_x) * 16;
    const int cblocks = a.Cin / 64, nk = 9 * cblocks;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(MT * N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[s])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = tmem_base;
    __shared__ int consumed;  // steps whose MMAs were issued (set by the issuer)
    bool ok = true;
    int issued = 0;
    if (tid == 0) {
        // producer: loads run up to S stages ahead of the MMAs
        const uint64_t pa = reinterpret_cast<uint64_t>(&ta), pw = reinterpret_cast<uint64_t>(&tw);
        for (int k = 0; k < nk; ++k) {
            const int s = k % S, tap = k / cblocks, cb = k - tap * cblocks;
            // slot s was last read by the MMAs of step k - S
            if (k >= S && !(ok = mbar_wait(smem_u32(&empty[s]), ((k / S) - 1) & 1, err, a.spin))) break;
            const int dy = (tap / 3 - 1) * a.dil, dx = (tap % 3 - 1) * a.dil;
            const uint32_t sa = sbase + s * STAGE, sb = sa + A_BYTES, bar = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(STAGE)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4, %5}], [%6];\n" ::"r"(sa),
                "l"(pa), "r"(cb * 64), "r"(x0 + dx), "r"(y0 + dy), "r"(b), "r"(bar)
                : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];\n" ::"r"(sb),
                "l"(pw), "r"(tap * a.Cin + cb * 64), "r"(0), "r"(bar)
                : "memory");
            issued = k + 1;
        }
    } else if (tid == 32) {
        // MMA issuer: each stage's MMAs as soon as its bytes land
        const uint32_t idesc = umma_idesc(128, N);
        int k = 0;
        for (; k < nk; ++k) {
            const int s = k % S;
            if (!(ok = mbar_wait(smem_u32(&full[s]), (k / S) & 1, err, a.spin))) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t sa = sbase + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t bd = umma_sdesc(sb + ks * 32);
                const uint32_t acc = (k > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
                for (int q = 0; q < MT; ++q) {
                    const uint64_t ad = umma_sdesc(sa + q * 128 * 128 + ks * 32);
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                            tmem + (uint32_t)(q * N)),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&empty[s])));
        }
        consumed = k;
    }
    const bool all_ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!all_ok && tid == 0) {
        // a wait gave up: let the loads this CTA issued and no MMA consumed land
        // before the shared memory is released (the default bound)
        for (int k = consumed; k < issued; ++k) mbar_wait(smem_u32(&full[k % S]), (k / S) & 1, err);
    }
    // every MMA issued has finished when the last issued step's commit arrives
    // (in issue order); after a give-up the MMAs still finish before the
    // tensor memory is freed
    ok = all_ok;
    const int nc = consumed;
    if (nc >= 1) {
        const uint32_t bar = smem_u32(&empty[(nc - 1) % S]), par = ((nc - 1) / S) & 1;
        bool w = ok && mbar_wait(bar, par, err, a.spin);
        if (!w) mbar_wait(bar, par, err);
        ok = __syncthreads_and((ok && w) ? 1 : 0) != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (ok) {
        // warp w reads lanes 32 (w % 4) .. of accumulator w / 4; accumulator
        // row r of window q is the pixel (y0 + 8 q + r / 16, x0 + r % 16)
        const int q = warp >> 2, r = ((warp & 3) << 5) + (tid & 31);
        const int py = y0 + 8 * q + (r >> 4), px = x0 + (r & 15);
        const long long m = ((long long)b * a.H + py) * a.W + px;
        const uint32_t lane = ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(q * N);
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(tmem + lane + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            uint32_t packed[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float f0 = __uint_as_float(v[2 * j]), f1 = __uint_as_float(v[2 * j + 1]);
                if (a.bias) {
                    f0 += a.bias[c0 + 2 * j];
                    f1 += a.bias[c0 + 2 * j + 1];
                }
                if (a.relu) {
                    f0 = fmaxf(f0, 0.f);
                    f1 = fmaxf(f1, 0.f);
                }
                __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
                packed[j] = *reinterpret_cast<uint32_t*>(&h);
            }
            uint4* dst = reinterpret_cast<uint4*>(a.y + m * N + c0);
            dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(MT * N));
}

struct WgradArgs {
    int B, H, W, Cin, Cout, dil;
    const bf16* x;   // layer input [B][H][W][Cin]
    const bf16* dy;  // gradient at the pre-activation [B][H][W][Cout]
    float* part;     // [splits][9 Cin][Cout]
    long long pchunk;
};

// dW[k][co] = sum_p X_patch[p][k] dY[p][co]: M = 9 Cin, N = Cout, reduction
// over pixels (split over blockIdx.z; partial sums reduced afterwards)
template <int BN>
__global__ void __launch_bounds__(128) k_conv_wgrad(WgradArgs a)
{
    constexpr int BM = 64, BP = 32, AS = BM + 8, BSTR = BN + 8;
    constexpr int WN = BN >= 64 ? 2 : 1, WM = 4 / WN, TM = BM / WM, TN = BN / WN;
    constexpr int MI = TM / 16, NI = TN / 8;
    __shared__ __align__(16) bf16 As[2][BP][AS];
    __shared__ __align__(16) bf16 Bs[2][BP][BSTR];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp / WN, wn = warp % WN;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int HW = a.H * a.W;
    const long long M = (long long)a.B * HW;
    const int K = 9 * a.Cin;
    const long long pbeg = (long long)blockIdx.z * a.pchunk;
    const long long pend = pbeg + a.pchunk < M ? pbeg + a.pchunk : M;
    float acc[MI][NI][4];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
    auto load = [&](int st, long long p0) {
        for (int v = tid; v < BP * (BM / 8); v += 128) {
            int row = v / (BM / 8), kg = v % (BM / 8);
            long long p = p0 + row;
            int k = m0 + kg * 8;
            const bf16* src = a.x;
            bool ok = false;
            if (p < pend && k < K) {
                int tap = k / a.Cin, ci = k - tap * a.Cin;
                int b = (int)(p / HW), rem = (int)(p - (long long)b * HW);
                int r = rem / a.W, c = rem - r * a.W;
                int rr = r + (tap / 3 - 1) * a.dil, cc = c + (tap % 3 - 1) * a.dil;
                if (rr >= 0 && rr < a.H && cc >= 0 && cc < a.W) {
                    src = a.x + (((long long)b * a.H + rr) * a.W + cc) * a.Cin + ci;
                    ok = true;
                }
            }
            cp_async16(&As[st][row][kg * 8], src, ok);
        }
        for (int v = tid; v < BP * (BN / 8); v += 128) {
            int row = v / (BN / 8), ng = v % (BN / 8);
            long long p = p0 + row;
            int n = n0 + ng * 8;
            bool ok = p < pend && n < a.Cout;
            cp_async16(&Bs[st][row][ng * 8], ok ? a.dy + p * a.Cout + n : a.dy, ok);
        }
        cp_async_commit();
    };
    const long long np = pend > pbeg ? (pend - pbeg + BP - 1) / BP : 0;
    if (np > 0) load(0, pbeg);
    for (long long pt = 0; pt < np; ++pt) {
        const int st = (int)(pt & 1);
        if (pt + 1 < np) {
            load(st ^ 1, pbeg + (pt + 1) * BP);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BP; kk += 16) {
            unsigned af[MI][4], bfr[NI][2];
#pragma unroll
            for (int i = 0; i < MI; ++i)
                ldsm_x4_t(af[i], &As[st][kk + (lane & 7) + ((lane >> 4) << 3)]
                                    [wm * TM + i * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int j = 0; j < NI; ++j) ldsm_x2_t(bfr[j], &Bs[st][kk + (lane & 15)][wn * TN + j * 8]);
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int j = 0; j < NI; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
    float* part = a.part + (size_t)blockIdx.z * K * a.Cout;
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j) {
            int n = n0 + wn * TN + j * 8 + 2 * t;
            if (n >= a.Cout) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int k = m0 + wm * TM + i * 16 + g + h * 8;
                if (k >= K) continue;
                part[(size_t)k * a.Cout + n] = acc[i][j][2 * h];
                part[(size_t)k * a.Cout + n + 1] = acc[i][j][2 * h + 1];
            }
        }
}

// grad[i] = sum over splits of part[s][i]  (fixed order: deterministic)
__global__ void k_sum_splits(const float* part, int splits, long long n, float* grad)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int q = 0; q < splits; ++q) s += part[(size_t)q * n + i];
    grad[i] = s;
}

// bias gradient: per channel sum over pixels (one block per channel)
__global__ void k_bias_grad(const bf16* dy, long long M, int C, float* grad)
{
    int c = blockIdx.x;
    float s = 0.f;
    for (long long p = threadIdx.x; p < M; p += blockDim.x) s += __bfloat162float(dy[p * C + c]);
    __shared__ float sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad[c] = sh[0];
}

// dYpre = dY where the layer's ReLU output is positive, else 0
__global__ void k_relu_bwd(const bf16* dy, const bf16* y, long long n, bf16* out)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = __bfloat162float(y[i]) > 0.f ? dy[i] : __float2bfloat16(0.f);
}

// loss = 1/2 mean over the M cells of (y[p][0] - t[p])^2, dY[p][0] = (y - t) / M,
// other channels 0; per-block partial sums of the loss (FP64)
__global__ void k_loss(const float* y32, int C, const float* t, long long M, bf16* dy, double* part)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double e2 = 0.0;
    if (p < M) {
        float e = y32[p * C] - t[p];
        e2 = 0.5 * (double)e * (double)e;
        dy[p * C] = __float2bfloat16(e / (float)M);
        for (int c = 1; c < C; ++c) dy[p * C + c] = __float2bfloat16(0.f);
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = e2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_sum_loss(const double* part, int n, long long count, double* loss)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *loss = s / (double)count;
}

struct LayerTab {
    long woff[kLayers], boff[kLayers];
    int cin[kLayers], cout[kLayers];
};

// BF16 copies of one FP32 parameter: the weights as stored (W[k][co], the
// mma.sync forward), K-major for the tensor-core forward (Wk[co][k]), and the
// flipped, transposed weights of the data gradient, [k'][ci] for mma.sync
// and K-major [ci][k'] for the tensor cores (k' = (8 - tap) Cout + co)
struct WeightCopies {
    bf16 *wb, *wt, *wk, *wtk;
};

__device__ __forceinline__ void write_copies(long long i, float p, const LayerTab& T, const WeightCopies& w)
{
    for (int l = 0; l < kLayers; ++l) {
        if (i >= T.woff[l] && i < T.boff[l]) {
            long long q = i - T.woff[l];
            int cin = T.cin[l], cout = T.cout[l];
            int co = (int)(q % cout);
            long long k = q / cout;
            int tap = (int)(k / cin), ci = (int)(k % cin);
            long long kp = (long long)(8 - tap) * cout + co;
            const bf16 pb = __float2bfloat16(p);
            w.wb[i] = pb;
            w.wt[T.woff[l] + kp * cin + ci] = pb;
            w.wk[T.woff[l] + (long long)co * 9 * cin + k] = pb;
            w.wtk[T.woff[l] + (long long)ci * 9 * cout + kp] = pb;
        }
    }
}

// Adam on the FP32 parameters; refreshes the BF16 weight copies
__global__ void k_adam(float* prm, float* m, float* v, const float* grad, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2, LayerTab T, WeightCopies w)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g = grad[i];
    float mi = b1 * m[i] + (1.f - b1) * g, vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    float p = prm[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    prm[i] = p;
    write_copies(i, p, T, w);
}

// the same refresh without an update (after loading parameters)
__global__ void k_refresh(const float* prm, long long n, LayerTab T, WeightCopies w)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    write_copies(i, prm[i], T, w);
}

// scale of every problem: max |u0| over its grid (1 when u0 is NULL or zero);
// one block per problem, max of non-negative doubles through their bit patterns
__global__ void k_scale(const double* u0, double* scale)
{
    const int b = blockIdx.x;
    unsigned long long m = 0ull;
    if (u0)
        for (long long k = threadIdx.x; k < (long long)kN * kN; k += blockDim.x) {
            unsigned long long v = (unsigned long long)__double_as_longlong(fabs(u0[(size_t)b * kN * kN + k]));
            m = v > m ? v : m;
        }
    __shared__ unsigned long long sh[256];
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w && sh[threadIdx.x + w] > sh[threadIdx.x]) sh[threadIdx.x] = sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double v = __longlong_as_double((long long)sh[0]);
        scale[b] = v > 0.0 ? v : 1.0;
    }
}

// features of a batch of 256 x 256 problems, one thread per cell (u0 nullable)
__global__ void k_features(int batch, const double* f, const double* b1, const double* b2,
                           const uint8_t* mask, const double* mu, const double* sigma,
                           const double* u0, const double* scale, bf16* x)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)batch * kHW * kHW) return;
    int b = (int)(q / (kHW * kHW)), rem = (int)(q % (kHW * kHW)), r = rem / kHW, c = rem % kHW;
    double s1 = 0, s2 = 0, sm = 0;
    size_t base = (size_t)b * kN * kN;
    bf16* o = x + q * kCin;
    for (int i = 0; i < kSub; ++i)
        for (int j = 0; j < kSub; ++j) {
            size_t k = base + (size_t)(r * kSub + i) * kN + (c * kSub + j);
            o[i * kSub + j] = __float2bfloat16((float)f[k]);
            o[16 + i * kSub + j] = __float2bfloat16(u0 ? (float)(u0[k] / scale[b]) : 0.f);
            s1 += b1[k];
            s2 += b2[k];
            sm += mask[k];
        }
    const double inv = 1.0 / (kSub * kSub);
    o[32] = __float2bfloat16((float)(s1 * inv));
    o[33] = __float2bfloat16((float)(s2 * inv));
    o[34] = __float2bfloat16((float)((log10(mu[b]) + 2.5) / 1.5));
    o[35] = __float2bfloat16((float)(sigma[b] - 1.0));
    o[36] = __float2bfloat16((float)(sm * inv));
    o[37] = o[38] = o[39] = __float2bfloat16(0.f);
}

// t[b][cell] = cell mean of (u - u0) / s_b, one thread per cell (u0 nullable)
__global__ void k_targets(int batch, const double* u, const double* u0, const double* scale,
                          float* t)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)batch * kHW * kHW) return;
    int b = (int)(q / (kHW * kHW)), rem = (int)(q % (kHW * kHW)), r = rem / kHW, c = rem % kHW;
    size_t base = (size_t)b * kN * kN;
    double sum = 0.0;
    for (int i = 0; i < kSub; ++i)
        for (int j = 0; j < kSub; ++j) {
            size_t k = base + (size_t)(r * kSub + i) * kN + (c * kSub + j);
            sum += u[k] - (u0 ? u0[k] : 0.0);
        }
    t[q] = (float)(sum / (kSub * kSub) / scale[b]);
}

// u = u0 + s * bilinear(y[..][0]) on the interior nodes, 0 elsewhere; cell
// centres at node 4 k + 1.5, clamped at the outer half cells (u0 nullable)
__global__ void k_upsample(const float* y, const double* u0, const double* scale,
                           const uint8_t* ntype, double* u)
{
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)kN * kN) return;
    int r = (int)(q / kN), c = (int)(q % kN);
    if (ntype[q] != adr::kInterior) {
        u[q] = 0.0;
        return;
    }
    double fy = (r - (kSub - 1) * 0.5) / kSub, fx = (c - (kSub - 1) * 0.5) / kSub;
    fy = fy < 0 ? 0 : (fy > kHW - 1 ? kHW - 1 : fy);
    fx = fx < 0 ? 0 : (fx > kHW - 1 ? kHW - 1 : fx);
    int y0 = (int)fy, x0 = (int)fx;
    if (y0 > kHW - 2) y0 = kHW - 2;
    if (x0 > kHW - 2) x0 = kHW - 2;
    double ly = fy - y0, lx = fx - x0;
    auto Y = [&](int rr, int cc) { return (double)y[((size_t)rr * kHW + cc) * kCout]; };
    double v = (1 - ly) * ((1 - lx) * Y(y0, x0) + lx * Y(y0, x0 + 1)) +
               ly * ((1 - lx) * Y(y0 + 1, x0) + lx * Y(y0 + 1, x0 + 1));
    u[q] = (u0 ? u0[q] : 0.0) + (scale ? *scale : 1.0) * v;
}

}  // namespace

// ------------------------------------------------------------------ handle

struct adr_cnn {
    int max_batch = 0, hw = kHW;
    cudaStream_t stream = nullptr;
    long P = 0;
    LayerTab T{};
    float *prm = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    bf16 *wb = nullptr, *wt = nullptr, *wk = nullptr, *wtk = nullptr;
    int* err = nullptr;  // a bounded wait of a tensor-core kernel gave up
    long long spin = 0;  // bound of those waits (adr_cnn_set_wait_limit; 0: default)
    bf16* act[kLayers] = {};  // post-activation outputs of layers 0..6 (bf16)
    float* y32 = nullptr;     // last layer output (fp32) [M][8]
    bf16 *dA = nullptr, *dB = nullptr, *dpre = nullptr;
    float* part = nullptr;
    long long part_size = 0;
    double* lpart = nullptr;
    double* loss = nullptr;
    long step = 0;
    std::vector<void*> owned;
};

namespace {

template <typename T>
adr_status cnn_alloc(adr_cnn* c, T** p, size_t n)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T) + 16);
    if (e != cudaSuccess) {
        adr::set_error(std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
        return ADR_ENOMEM;
    }
    c->owned.push_back(q);
    *p = static_cast<T*>(q);
    return ADR_OK;
}

template <int N>
constexpr int tc_smem_bytes()
{
    return 2 * (128 * 128 + N * 128) + 1024;
}

// the driver's tensor-map encoder, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* q = nullptr;
        cudaDriverEntryPointQueryResult res = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &res) ==
                cudaSuccess &&
            res == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(q);
        else
            cudaGetLastError();
    }
    return fn;
}

// tensor maps of a convolution's input [B][H][W][Cin] (box: 64 channels x 16 x
// 8 pixels) and K-major weights [N][9 Cin] (box: 64 x N), 128-byte swizzle;
// false when the driver refuses them (the caller takes another kernel)
bool conv_tensor_maps(const ConvArgs& a, const bf16* wk, CUtensorMap* ta, CUtensorMap* tw)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t C = (cuuint64_t)a.Cin, K = 9 * C;
    cuuint64_t dA[4] = {C, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.B};
    cuuint64_t sA[3] = {C * 2, C * 2 * a.W, C * 2 * a.W * a.H};
    cuuint32_t bA[4] = {64, 16, 8 * kTmaMT, 1}, e4[4] = {1, 1, 1, 1};
    if (enc(ta, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(a.x), dA, sA, bA, e4,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    cuuint64_t dW[2] = {K, (cuuint64_t)a.Cout};
    cuuint64_t sW[1] = {K * 2};
    cuuint32_t bW[2] = {64, (cuuint32_t)a.Cout}, e2[2] = {1, 1};
    return enc(tw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(wk), dW, sW, bW, e2,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor-core paths for 64 or 128 output channels with a BF16 output (wk: the
// K-major weights): TMA-fed for inputs of a multiple of 64 channels on 8 x 16
// pixel windows, cp.async-fed otherwise; mma.sync for the rest
void launch_conv(cudaStream_t st, const ConvArgs& a, const bf16* wk = nullptr, int* err = nullptr)
{
    long long M = (long long)a.B * a.H * a.W;
    if (wk && err && a.y && !a.y32 && (a.Cout == 64 || a.Cout == 128) && a.Cin % 64 == 0 &&
        a.H % (8 * kTmaMT) == 0 && a.W % 16 == 0) {
        CUtensorMap ta, tw;
        if (conv_tensor_maps(a, wk, &ta, &tw)) {
            ConvArgs t = a;
            t.w = wk;
            const unsigned blocks = (unsigned)(a.B * (a.H / (8 * kTmaMT)) * (a.W / 16));
            if (a.Cout == 64)
                k_conv_tma<64><<<blocks, TmaConv<64>::THREADS, TmaConv<64>::SMEM, st>>>(ta, tw, t, err);
            else
                k_conv_tma<128><<<blocks, TmaConv<128>::THREADS, TmaConv<128>::SMEM, st>>>(ta, tw, t, err);
            return;
        }
    }
    if (wk && err && a.y && !a.y32 && (a.Cout == 64 || a.Cout == 128)) {
        ConvArgs t = a;
        t.w = wk;
        const unsigned blocks = (unsigned)((M + 127) / 128);
        if (a.Cout == 64) k_conv_tc<64><<<blocks, 128, tc_smem_bytes<64>(), st>>>(t, err);
        else k_conv_tc<128><<<blocks, 128, tc_smem_bytes<128>(), st>>>(t, err);
        return;
    }
    dim3 grid((unsigned)((M + 127) / 128), 1);
    if (a.Cout >= 64) {
        grid.y = (a.Cout + 63) / 64;
        k_conv_fwd<64><<<grid, 256, 0, st>>>(a);
    } else if (a.Cout % 16 == 0) {
        grid.y = a.Cout / 16;
        k_conv_fwd<16><<<grid, 256, 0, st>>>(a);
    } else {
        grid.y = (a.Cout + 7) / 8;
        k_conv_fwd<8><<<grid, 256, 0, st>>>(a);
    }
}

// forward of a batch: act[0..6] bf16, y32 of the last layer
adr_status cnn_forward(adr_cnn* c, int batch, const bf16* x)
{
    const bf16* in = x;
    for (int l = 0; l < kLayers; ++l) {
        ConvArgs a{};
        a.B = batch;
        a.H = a.W = c->hw;
        a.Cin = kCh[l];
        a.Cout = kCh[l + 1];
        a.dil = kDil[l];
        a.x = in;
        a.w = c->wb + c->T.woff[l];
        a.bias = c->prm + c->T.boff[l];
        a.relu = l < kLayers - 1;
        a.spin = c->spin;
        if (l < kLayers - 1) a.y = c->act[l];
        else a.y32 = c->y32;
        launch_conv(c->stream, a, c->wk + c->T.woff[l], c->err);
        in = c->act[l];
    }
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status cnn_backward(adr_cnn* c, int batch, const bf16* x, const float* t)
{
    cudaStream_t st = c->stream;
    const long long M = (long long)batch * c->hw * c->hw;
    int nb = (int)((M + 255) / 256);
    bf16* dy = c->dA;
    k_loss<<<nb, 256, 0, st>>>(c->y32, kCout, t, M, dy, c->lpart);
    k_sum_loss<<<1, 1, 0, st>>>(c->lpart, nb, M, c->loss);
    for (int l = kLayers - 1; l >= 0; --l) {
        const int cin = kCh[l], cout = kCh[l + 1];
        const bf16* dyp = dy;
        if (l < kLayers - 1) {
            k_relu_bwd<<<(int)((M * cout + 255) / 256), 256, 0, st>>>(dy, c->act[l], M * cout, c->dpre);
            dyp = c->dpre;
        }
        const bf16* xin = l == 0 ? x : c->act[l - 1];
        // weight gradient, split over pixels
        WgradArgs w{};
        w.B = batch;
        w.H = w.W = c->hw;
        w.Cin = cin;
        w.Cout = cout;
        w.dil = kDil[l];
        w.x = xin;
        w.dy = dyp;
        w.part = c->part;
        long long K = 9LL * cin;
        int splits = (int)std::min<long long>(64, (M + 1023) / 1024);
        if (splits < 1) splits = 1;
        while ((long long)splits * K * cout > c->part_size) splits--;
        w.pchunk = ((M + splits - 1) / splits + 31) / 32 * 32;
        splits = (int)((M + w.pchunk - 1) / w.pchunk);
        dim3 grid((unsigned)((K + 63) / 64), 1, (unsigned)splits);
        if (cout >= 64) {
            grid.y = (cout + 63) / 64;
            k_conv_wgrad<64><<<grid, 128, 0, st>>>(w);
        } else if (cout % 16 == 0) {
            grid.y = cout / 16;
            k_conv_wgrad<16><<<grid, 128, 0, st>>>(w);
        } else {
            grid.y = (cout + 7) / 8;
            k_conv_wgrad<8><<<grid, 128, 0, st>>>(w);
        }
        long long nw = K * cout;
        k_sum_splits<<<(int)((nw + 255) / 256), 256, 0, st>>>(c->part, splits, nw, c->grad + c->T.woff[l]);
        k_bias_grad<<<cout, 256, 0, st>>>(dyp, M, cout, c->grad + c->T.boff[l]);
        if (l > 0) {
            // data gradient: correlation with the flipped, transposed weights
            ConvArgs a{};
            a.B = batch;
            a.H = a.W = c->hw;
            a.Cin = cout;
            a.Cout = cin;
            a.dil = kDil[l];
            a.x = dyp;
            a.w = c->wt + c->T.woff[l];
            a.spin = c->spin;
            a.y = dy == c->dA ? c->dB : c->dA;
            launch_conv(st, a, c->wtk + c->T.woff[l], c->err);
            dy = a.y;
        }
    }
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

// a bounded wait gave up: clear the flag and report it
adr_status report_timeout(adr_cnn* c)
{
    cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
    adr::set_error("a tensor-core kernel gave up waiting (bounded mbarrier wait); its outputs are not valid");
    return ADR_ETIMEOUT;
}

}  // namespace

extern "C" {

long adr_cnn_num_params(void) { return param_offset(kLayers, false); }

adr_status adr_cnn_set_wait_limit(adr_cnn* c, long long spins)
{
    if (!c || spins < 0) {
        adr::set_error("adr_cnn_set_wait_limit: NULL handle or negative bound");
        return ADR_EINVAL;
    }
    c->spin = spins;
    return ADR_OK;
}

adr_status adr_cnn_sync(adr_cnn* c)
{
    if (!c) {
        adr::set_error("adr_cnn_sync: NULL handle");
        return ADR_EINVAL;
    }
    int e = 0;
    ADR_CUDA_TRY(cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    ADR_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return e ? report_timeout(c) : ADR_OK;
}

void adr_cnn_destroy(adr_cnn* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (void* q : c->owned) cudaFree(q);
    delete c;
}

adr_status adr_cnn_set_params(adr_cnn* c, const float* host)
{
    if (!c || !host) {
        adr::set_error("NULL argument");
        return ADR_EINVAL;
    }
    ADR_CUDA_TRY(cudaMemcpyAsync(c->prm, host, sizeof(float) * c->P, cudaMemcpyHostToDevice, c->stream));
    ADR_CUDA_TRY(cudaMemsetAsync(c->m, 0, sizeof(float) * c->P, c->stream));
    ADR_CUDA_TRY(cudaMemsetAsync(c->v, 0, sizeof(float) * c->P, c->stream));
    c->step = 0;
    k_refresh<<<(int)((c->P + 255) / 256), 256, 0, c->stream>>>(c->prm, c->P, c->T,
                                                                WeightCopies{c->wb, c->wt, c->wk, c->wtk});
    ADR_CUDA_TRY(cudaGetLastError());
    ADR_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return ADR_OK;
}

adr_status adr_cnn_get_params(adr_cnn* c, float* host)
{
    if (!c || !host) {
        adr::set_error("NULL argument");
        return ADR_EINVAL;
    }
    ADR_CUDA_TRY(cudaMemcpyAsync(host, c->prm, sizeof(float) * c->P, cudaMemcpyDeviceToHost, c->stream));
    ADR_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return ADR_OK;
}

adr_status adr_cnn_create(int max_batch, const float* params, void* stream, adr_cnn** out)
{
    if (!out || max_batch < 1 || !params) {
        adr::set_error("adr_cnn_create needs max_batch >= 1, initial parameters and an output");
        return ADR_EINVAL;
    }
    *out = nullptr;
    adr_cnn* c = new (std::nothrow) adr_cnn;
    if (!c) return ADR_ENOMEM;
    c->max_batch = max_batch;
    c->stream = static_cast<cudaStream_t>(stream);
    c->P = param_offset(kLayers, false);
    for (int l = 0; l < kLayers; ++l) {
        c->T.woff[l] = param_offset(l, false);
        c->T.boff[l] = param_offset(l, true);
        c->T.cin[l] = kCh[l];
        c->T.cout[l] = kCh[l + 1];
    }
    const long long M = (long long)max_batch * c->hw * c->hw;
    adr_status s = ADR_OK;
    auto fail = [&](adr_status st) {
        adr_cnn_destroy(c);
        return st;
    };
    if ((s = cnn_alloc(c, &c->prm, c->P)) || (s = cnn_alloc(c, &c->m, c->P)) ||
        (s = cnn_alloc(c, &c->v, c->P)) || (s = cnn_alloc(c, &c->grad, c->P)) ||
        (s = cnn_alloc(c, &c->wb, c->P)) || (s = cnn_alloc(c, &c->wt, c->P)) ||
        (s = cnn_alloc(c, &c->wk, c->P)) || (s = cnn_alloc(c, &c->wtk, c->P)) ||
        (s = cnn_alloc(c, &c->err, 1)) ||
        (s = cnn_alloc(c, &c->y32, M * kCout)) || (s = cnn_alloc(c, &c->dA, M * 128)) ||
        (s = cnn_alloc(c, &c->dB, M * 128)) || (s = cnn_alloc(c, &c->dpre, M * 128)) ||
        (s = cnn_alloc(c, &c->lpart, (M + 255) / 256 + 1)) || (s = cnn_alloc(c, &c->loss, 1)))
        return fail(s);
    for (int l = 0; l < kLayers - 1; ++l)
        if ((s = cnn_alloc(c, &c->act[l], M * kCh[l + 1]))) return fail(s);
    c->part_size = 64LL * 9 * 128 * 128;
    if ((s = cnn_alloc(c, &c->part, c->part_size))) return fail(s);
    ADR_CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    // the tensor-core kernels use more than 48 KB of shared memory (per device)
    ADR_CUDA_TRY(cudaFuncSetAttribute(k_conv_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tc_smem_bytes<64>()));
    ADR_CUDA_TRY(cudaFuncSetAttribute(k_conv_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tc_smem_bytes<128>()));
    ADR_CUDA_TRY(cudaFuncSetAttribute(k_conv_tma<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TmaConv<64>::SMEM));
    ADR_CUDA_TRY(cudaFuncSetAttribute(k_conv_tma<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      TmaConv<128>::SMEM));
    if ((s = adr_cnn_set_params(c, params))) return fail(s);
    *out = c;
    return ADR_OK;
}

adr_status adr_cnn_features(int batch, int n, const double* f, const double* b1, const double* b2,
                            const uint8_t* mask, const double* mu, const double* sigma,
                            const double* u0, uint16_t* x, double* scale, void* stream)
{
    if (batch < 1 || n != kN || !f || !b1 || !b2 || !mask || !mu || !sigma || !x || !scale) {
        adr::set_error("adr_cnn_features: bad arguments (the network reads 256 x 256 grids)");
        return ADR_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_scale<<<batch, 256, 0, st>>>(u0, scale);
    long long q = (long long)batch * kHW * kHW;
    k_features<<<(int)((q + 255) / 256), 256, 0, st>>>(batch, f, b1, b2, mask, mu, sigma, u0, scale,
                                                       reinterpret_cast<bf16*>(x));
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status adr_cnn_targets(int batch, int n, const double* u, const double* u0,
                           const double* scale, float* t, void* stream)
{
    if (batch < 1 || n != kN || !u || !scale || !t) {
        adr::set_error("adr_cnn_targets: bad arguments (the network reads 256 x 256 grids)");
        return ADR_EINVAL;
    }
    long long q = (long long)batch * kHW * kHW;
    k_targets<<<(int)((q + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(batch, u, u0,
                                                                                    scale, t);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}

adr_status adr_cnn_forward(adr_cnn* c, int batch, const uint16_t* x, float* y)
{
    if (!c || batch < 1 || batch > c->max_batch || !x || !y) {
        adr::set_error("adr_cnn_forward: bad arguments");
        return ADR_EINVAL;
    }
    TRY_S(cnn_forward(c, batch, reinterpret_cast<const bf16*>(x)));
    const long long M = (long long)batch * c->hw * c->hw;
    ADR_CUDA_TRY(cudaMemcpyAsync(y, c->y32, sizeof(float) * M * kCout, cudaMemcpyDeviceToDevice,
                                 c->stream));
    return ADR_OK;
}

adr_status adr_cnn_loss_grad(adr_cnn* c, int batch, const uint16_t* x, const float* t, float* grad,
                             double* loss)
{
    if (!c || batch < 1 || batch > c->max_batch || !x || !t) {
        adr::set_error("adr_cnn_loss_grad: bad arguments");
        return ADR_EINVAL;
    }
    const bf16* xb = reinterpret_cast<const bf16*>(x);
    TRY_S(cnn_forward(c, batch, xb));
    TRY_S(cnn_backward(c, batch, xb, t));
    if (grad)
        ADR_CUDA_TRY(cudaMemcpyAsync(grad, c->grad, sizeof(float) * c->P, cudaMemcpyDeviceToDevice,
                                     c->stream));
    if (loss) {
        int e = 0;
        ADR_CUDA_TRY(cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        ADR_CUDA_TRY(cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        ADR_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (e) return report_timeout(c);
    }
    return ADR_OK;
}

adr_status adr_cnn_train_step(adr_cnn* c, int batch, const uint16_t* x, const float* t, float lr,
                              double* loss)
{
    if (!c || batch < 1 || batch > c->max_batch || !x || !t || !(lr > 0.f)) {
        adr::set_error("adr_cnn_train_step: bad arguments");
        return ADR_EINVAL;
    }
    const bf16* xb = reinterpret_cast<const bf16*>(x);
    TRY_S(cnn_forward(c, batch, xb));
    TRY_S(cnn_backward(c, batch, xb, t));
    c->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - powf(b1, (float)c->step), c2 = 1.f - powf(b2, (float)c->step);
    k_adam<<<(int)((c->P + 255) / 256), 256, 0, c->stream>>>(
        c->prm, c->m, c->v, c->grad, c->P, lr, b1, b2, 1e-8f, c1, c2, c->T,
        WeightCopies{c->wb, c->wt, c->wk, c->wtk});
    ADR_CUDA_TRY(cudaGetLastError());
    if (loss) {
        int e = 0;
        ADR_CUDA_TRY(cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        ADR_CUDA_TRY(cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        ADR_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (e) return report_timeout(c);
    }
    return ADR_OK;
}

}  // extern "C"

namespace adr {
// forward of a batch on stream st (a problem's stream): ordered after the
// network's pending work and before its later work by events both ways
adr_status cnn_forward_on(adr_cnn* c, int batch, const uint16_t* x, float* y, cudaStream_t st)
{
    if (!c || batch < 1 || batch > c->max_batch || !x || !y) {
        set_error("warm start: bad network call");
        return ADR_EINVAL;
    }
    cudaEvent_t ev = nullptr;
    ADR_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    const cudaStream_t own = c->stream;
    adr_status s = ADR_OK;
    cudaError_t e = cudaEventRecord(ev, own);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    if (e != cudaSuccess) s = cuda_fail(e, "warm start: stream order");
    if (s == ADR_OK) {
        c->stream = st;
        s = adr_cnn_forward(c, batch, x, y);
        c->stream = own;
    }
    if (s == ADR_OK) {
        e = cudaEventRecord(ev, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(own, ev, 0);
        if (e != cudaSuccess) s = cuda_fail(e, "warm start: stream order");
    }
    cudaEventDestroy(ev);
    return s;
}

// one prediction [64][64][8] around u0 to the handle's 256 x 256 grid
adr_status launch_cnn_upsample(Problem* p, const float* y, const double* u0, const double* scale,
                               double* u)
{
    long long N = p->N;
    k_upsample<<<(int)((N + 255) / 256), 256, 0, p->stream>>>(y, u0, scale, p->ntype, u);
    ADR_CUDA_TRY(cudaGetLastError());
    return ADR_OK;
}
}  // namespace adr
