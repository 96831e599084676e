// Warm-start network on the GPU: BF16 tensor-core matrix products (tcgen05
// MMA with the accumulator in tensor memory, FP32 accumulation) with fused
// epilogues, SiLU hidden layers, mean-squared-error loss, backpropagation
// and Adam, all in the kernels below.  Contract in include/lbm_mlp.h.
//
// Every product is C[M][N] = A[M][K] * Bt[N][K]^T with both operands stored
// K-contiguous ("NT"):
//   forward     act_out[B][N]  = act_in[B][K]  * Wt[N][K]^T   (+ bias, SiLU)
//   input grad  g_in[B][K]     = g_out[B][N]   * W[K][N]^T    (x SiLU'(pre))
//   weight grad dWt[N][K]      = g_out^T[N][B] * act_in^T[K][B]^T
// so each layer keeps its weights in both layouts (Wt and W) and the
// backward pass transposes activations and output gradients.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/lbm_mlp.h"

namespace {

#ifndef LBM_MLP_MMA_SYNC
#define LBM_MLP_MMA_SYNC 0  // 1: the warp-level mma.sync products instead of tcgen05 (for comparison)
#endif

using bf16 = __nv_bfloat16;
constexpr int K0 = 16;       // padded input width

enum { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_DX = 2, EPI_DW = 3 };

struct Epi {
    const float *bias;   // EPI_HIDDEN, EPI_OUT
    float *pre;          // EPI_HIDDEN: pre-activation out
    bf16 *out_bf;        // EPI_HIDDEN: SiLU(pre); EPI_DX: gradient (bf16)
    float *out_f;        // EPI_OUT: y; EPI_DX: gradient (fp32); EPI_DW: dWt
    const float *pre_in; // EPI_DX: pre-activation of the layer below
};

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

#if LBM_MLP_MMA_SYNC
constexpr int TM = 64, TN = 64, TK = 32;

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M][N] = A[M][K] * Bt[N][K]^T; M, N multiples of 16, K a multiple of 16.
// 128 threads: 2 x 2 warps, each a 32 x 32 sub-tile of the 64 x 64 block tile.
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_nt(const bf16 *__restrict__ A, const bf16 *__restrict__ Bt, int M,
                                                 int N, int K, Epi e) {
    __shared__ __align__(16) bf16 As[TM][TK + 8];
    __shared__ __align__(16) bf16 Bs[TN][TK + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int k = 0; k < 4; k++) acc[i][j][k] = 0.f;
    for (int k0 = 0; k0 < K; k0 += TK) {
        // each thread loads 16 bf16 (two 16-byte chunks) of A and of Bt
        {
            const int r = tid >> 1, c = (tid & 1) * 16;
            uint4 va0 = make_uint4(0, 0, 0, 0), va1 = va0, vb0 = va0, vb1 = va0;
            if (m0 + r < M && k0 + c < K) {
                const uint4 *p = reinterpret_cast<const uint4 *>(A + (size_t)(m0 + r) * K + k0 + c);
                va0 = p[0];
                va1 = p[1];
            }
            if (n0 + r < N && k0 + c < K) {
                const uint4 *p = reinterpret_cast<const uint4 *>(Bt + (size_t)(n0 + r) * K + k0 + c);
                vb0 = p[0];
                vb1 = p[1];
            }
            *reinterpret_cast<uint4 *>(&As[r][c]) = va0;
            *reinterpret_cast<uint4 *>(&As[r][c + 8]) = va1;
            *reinterpret_cast<uint4 *>(&Bs[r][c]) = vb0;
            *reinterpret_cast<uint4 *>(&Bs[r][c + 8]) = vb1;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk += 16) {
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int r = wm * 32 + i * 16 + g;
                a[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * t]);
                a[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * t]);
                a[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 8 + 2 * t]);
                a[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int c = wn * 32 + j * 8 + g;
                b[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * t]);
                b[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int row = m0 + wm * 32 + i * 16 + g + 8 * h;
                const int col = n0 + wn * 32 + j * 8 + 2 * t;
                if (row >= M || col >= N) continue;
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    const float v = acc[i][j][2 * h + q];
                    const size_t idx = (size_t)row * N + col + q;
                    if (EPI == EPI_HIDDEN) {
                        const float z = v + e.bias[col + q];
                        e.pre[idx] = z;
                        e.out_bf[idx] = __float2bfloat16_rn(silu_f(z));
                    } else if (EPI == EPI_OUT) {
                        e.out_f[idx] = v + e.bias[col + q];
                    } else if (EPI == EPI_DX) {
                        const float gr = v * silu_grad_f(e.pre_in[idx]);
                        e.out_f[idx] = gr;
                        e.out_bf[idx] = __float2bfloat16_rn(gr);
                    } else {
                        e.out_f[idx] = v;
                    }
                }
            }
}
#endif  // LBM_MLP_MMA_SYNC

// ---------------------------------------------------------------------------
// tcgen05 product C[M][N] = A[M][K] * Bt[N][K]^T (BF16 operands, FP32
// accumulator in tensor memory).  One CTA of 128 threads per 128 x NT tile of
// C (NT = 32 or 16 columns).  The K range is walked in chunks of 64 through
// two shared-memory stages: the four warps start the asynchronous copies
// (cp.async, 16 bytes each) of chunk j + 1's A tile (128 rows) and B tile
// (NT rows) into stage (j + 1) % 2 before the tensor core works on chunk j.  The tiles are laid out in the canonical
// no-swizzle K-major form of the tensor-core descriptors: 8-row x 16-byte
// core matrices, element (r, k) of a tile at byte
// ((r / 8) * 8 + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, so that the core
// matrix next in K is 128 bytes on (the descriptor's leading-dimension
// offset) and the next 8-row group 1024 bytes on (its stride offset).  One
// thread issues one MMA (M = 128, N = NT, K = 16) per 16 columns of the chunk
// and commits them to the stage's mbarrier, which the copy of chunk j + 2
// waits for.  After the last chunk each warp reads its 32 rows of the
// accumulator (tensor-memory lanes 32 w .. 32 w + 31) with tcgen05.ld and
// applies the epilogue, 16 consecutive columns of a row per thread with
// 16-byte loads and stores.  Rows >= M and columns >= N are computed from zeros
// and not stored.  Every wait is bounded: on a time-out the kernel sets
// *err, waits (bounded) for its own MMAs, frees its tensor memory and leaves.
constexpr int TC_M = 128, TC_K = 64;
constexpr int TC_THREADS = 128;
constexpr long long TC_SPIN = 1ll << 22;  // mbarrier polls before a time-out

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, the fixed 0b001 at bits 46-48, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28
template <int NT> __device__ __forceinline__ uint32_t tc_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (long long it = 0; it < TC_SPIN; it++) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\n"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Epilogue of 16 consecutive columns col .. col + 15 of one row (col and N
// multiples of 16): 16-byte vector loads and stores.
template <int EPI> __device__ __forceinline__ void epi_store16(const Epi &e, int row, int col, int N, const uint32_t *r) {
    const size_t idx = (size_t)row * N + col;
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
    if (EPI == EPI_HIDDEN || EPI == EPI_OUT) {
        const float4 *b4 = reinterpret_cast<const float4 *>(e.bias + col);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float4 b = b4[q];
            v[4 * q] += b.x;
            v[4 * q + 1] += b.y;
            v[4 * q + 2] += b.z;
            v[4 * q + 3] += b.w;
        }
    }
    if (EPI == EPI_DX) {
        const float4 *p4 = reinterpret_cast<const float4 *>(e.pre_in + idx);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float4 z = p4[q];
            v[4 * q] *= silu_grad_f(z.x);
            v[4 * q + 1] *= silu_grad_f(z.y);
            v[4 * q + 2] *= silu_grad_f(z.z);
            v[4 * q + 3] *= silu_grad_f(z.w);
        }
    }
    float *of = EPI == EPI_HIDDEN ? e.pre : e.out_f;
    float4 *o4 = reinterpret_cast<float4 *>(of + idx);
#pragma unroll
    for (int q = 0; q < 4; q++) o4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    if (EPI == EPI_HIDDEN || EPI == EPI_DX) {
        uint32_t w[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float a = EPI == EPI_HIDDEN ? silu_f(v[2 * q]) : v[2 * q];
            const float b = EPI == EPI_HIDDEN ? silu_f(v[2 * q + 1]) : v[2 * q + 1];
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            w[q] = *reinterpret_cast<const uint32_t *>(&h);
        }
        uint4 *b4 = reinterpret_cast<uint4 *>(e.out_bf + idx);
        b4[0] = make_uint4(w[0], w[1], w[2], w[3]);
        b4[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

template <int EPI, int NT>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(const bf16 *__restrict__ A, const bf16 *__restrict__ Bt,
                                                        int M, int N, int K, Epi e, int *err) {
    constexpr int TMEM_COLS = 32;  // NT <= 32 accumulator columns (the minimum allocation)
    constexpr int A_BYTES = TC_M * TC_K * 2, B_BYTES = NT * TC_K * 2;
    static_assert(NT == 16 || NT == 32, "tile width");
    __shared__ __align__(1024) uint8_t sA[2][A_BYTES];
    __shared__ __align__(1024) uint8_t sB[2][B_BYTES];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * NT;
    const uint32_t bar_a[2] = {smem_u32(&bar[0]), smem_u32(&bar[1])};
    if (tid == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a[0]));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a[1]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tc_idesc<NT>();
    const int nchunk = (K + TC_K - 1) / TC_K;
    // asynchronous copy of chunk j into stage j % 2 (rows or columns past the
    // matrix are zero-filled): A tile 128 rows x 8 pieces of 16 bytes, B tile NT rows
    auto copy_chunk = [&](int j) {
        const int st = j & 1, k0 = j * TC_K;
        const uint32_t a_s = smem_u32(sA[st]), b_s = smem_u32(sB[st]);
        for (int q = tid; q < (TC_M + NT) * (TC_K / 8); q += TC_THREADS) {
            const bool isA = q < TC_M * (TC_K / 8);
            const int qq = isA ? q : q - TC_M * (TC_K / 8);
            const int r = qq >> 3, kc = qq & 7;
            const int grow = (isA ? m0 : n0) + r, gk = k0 + kc * 8;
            const bool valid = grow < (isA ? M : N) && gk < K;
            const bf16 *src = valid ? (isA ? A : Bt) + (size_t)grow * K + gk : A;
            cp_async16((isA ? a_s : b_s) + (uint32_t)(((r >> 3) * 8 + kc) * 128 + (r & 7) * 16), src, valid);
        }
    };
    bool ok = true;
    int last = -1;  // the last chunk whose MMAs were committed
    copy_chunk(0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int j = 0; j < nchunk && ok; j++) {
        const int st = j & 1, k0 = j * TC_K;
        if (j + 1 < nchunk) {
            // stage (j + 1) % 2 was last read by the MMAs of chunk j - 1
            if (j >= 1 && !mbar_wait(bar_a[(j + 1) & 1], ((j - 1) >> 1) & 1)) atomicExch(&failed, 1);
            if (!failed) copy_chunk(j + 1);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // chunk j has landed
        // make the copies visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (failed) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_base = smem_u32(sA[st]), b_base = smem_u32(sB[st]);
            const int nk = min(TC_K / 16, (K - k0 + 15) / 16);
            for (int kk = 0; kk < nk; kk++) {
                const uint64_t ad = tc_desc(a_base + kk * 256, 128, 1024);
                const uint64_t bd = tc_desc(b_base + kk * 256, 128, 1024);
                const uint32_t acc = (k0 > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\n"
                    "setp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar_a[st])
                         : "memory");
        }
        last = j;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy outlives the kernel
    // the last commit completes when all MMAs issued before it have completed
    if (last >= 0 && !mbar_wait(bar_a[last & 1], (last >> 1) & 1)) atomicExch(&failed, 1);
    __syncthreads();
    if (failed) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // epilogue: warp w holds rows 32 w .. 32 w + 31 (tensor-memory lanes), 16 columns per load
        const int row = m0 + warp * 32 + (tid & 31);
#pragma unroll
        for (int c0 = 0; c0 < NT; c0 += 16) {
            uint32_t r[16];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M && n0 + c0 < N) epi_store16<EPI>(e, row, n0 + c0, N, r);  // N is a multiple of 16
        }
    } else {
        if (tid == 0) atomicExch(err, 1);
        // the MMAs still in flight (bounded; their commit was the last one)
        if (last >= 0) mbar_wait(bar_a[last & 1], (last >> 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

__global__ void k_transpose_bf16(const bf16 *__restrict__ in, bf16 *__restrict__ out, int R, int C) {
    __shared__ bf16 tile[32][33];
    const int c = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8)
        if (r0 + k < R && c < C) tile[k][threadIdx.x] = in[(size_t)(r0 + k) * C + c];
    __syncthreads();
    const int r = r0 + threadIdx.x, c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8)
        if (c0 + k < C && r < R) out[(size_t)(c0 + k) * R + r] = tile[threadIdx.x][k];
}

// Gathers minibatch rows into the padded BF16 input and the FP32 target.
__global__ void k_gather_batch(const float *__restrict__ xd, const float *__restrict__ td,
                               const int32_t *__restrict__ idx, int batch, int n_in, int n_out, bf16 *x_bf,
                               float *t) {
    const int b = blockIdx.x, j = threadIdx.x;
    const int r = idx[b];
    if (j < K0) x_bf[(size_t)b * K0 + j] = __float2bfloat16_rn(j < n_in ? xd[(size_t)r * n_in + j] : 0.f);
    for (int k = j; k < n_out; k += blockDim.x) t[(size_t)b * n_out + k] = td[(size_t)r * n_out + k];
}

// d loss / d y for the mean squared error, and per-row partial sums of the loss.
__global__ void k_mse_grad(const float *__restrict__ y, const float *__restrict__ t, int batch, int n_out,
                           float *g_f, bf16 *g_bf, float *row_loss) {
    const int b = blockIdx.x;
    float s = 0.f;
    const float scale = 2.f / (float)(batch * n_out);
    for (int k = threadIdx.x; k < n_out; k += blockDim.x) {
        const size_t i = (size_t)b * n_out + k;
        const float d = y[i] - t[i];
        s += d * d;
        g_f[i] = scale * d;
        g_bf[i] = __float2bfloat16_rn(scale * d);
    }
    __shared__ float red[64];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) row_loss[b] = red[0];
}

__global__ void k_sum_loss(const float *row_loss, int batch, int n_out, float *loss) {
    __shared__ float red[256];
    float s = 0.f;
    for (int b = threadIdx.x; b < batch; b += 256) s += row_loss[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (float)(batch * n_out);
}

// db[n] = sum over the batch of g[b][n]; one thread per column, fixed order.
__global__ void k_bias_grad(const float *__restrict__ g, int batch, int n, float *db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float s = 0.f;
    for (int b = 0; b < batch; b++) s += g[(size_t)b * n + c];
    db[c] = s;
}

// Copies a (rows x cols_pad) FP32 block into (rows x cols) at dst (drops padding).
__global__ void k_unpad(const float *__restrict__ src, int rows, int cols_pad, int cols, float *dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    dst[i] = src[(size_t)(i / cols) * cols_pad + i % cols];
}

// Master FP32 layer weights (flat, n_out x n_in) -> BF16 Wt (n_out x K pad) and W (K pad x n_out).
__global__ void k_refresh_bf16(const float *__restrict__ wt, int n_out, int n_in, int kpad, bf16 *Wt_bf,
                               bf16 *W_bf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_out * kpad) return;
    const int r = i / kpad, c = i % kpad;
    const bf16 v = __float2bfloat16_rn(c < n_in ? wt[(size_t)r * n_in + c] : 0.f);
    Wt_bf[i] = v;
    W_bf[(size_t)c * n_out + r] = v;
}

__global__ void k_adam(float *theta, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

struct lbm_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_in = 0, n_out = 0, hidden = 0, n_layers = 0, max_batch = 0;
    std::vector<int> nin, nout, kpad;     // per layer
    std::vector<int64_t> woff, boff;      // offsets into the flat parameter vector
    int64_t np = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    std::vector<bf16 *> Wt, W;            // per layer
    std::vector<bf16 *> act;              // act[l]: input of layer l (B x kpad[l]) ; act[L] unused
    std::vector<float *> pre;             // pre-activation of hidden layer l (B x nout[l])
    std::vector<bf16 *> actT;             // transposed inputs (kpad[l] x B)
    float *y = nullptr, *t = nullptr, *row_loss = nullptr, *losses = nullptr;
    std::vector<float *> gf;              // gradient w.r.t. layer l output (B x nout[l]), fp32
    std::vector<bf16 *> gbf, gT;          // bf16 copy and transpose
    float *dw = nullptr;                  // padded dWt scratch (max nout x kpad)
    float *xd = nullptr, *td = nullptr;   // training set
    int n_data = 0;
    int32_t *idx = nullptr;
    int64_t adam_steps = 0;
    int *err = nullptr;                   // device: set by a tensor-core product that timed out
    std::vector<void *> allocs;
};

namespace {

template <class T> cudaError_t dal(lbm_mlp *h, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, (n ? n : 1) * sizeof(T));
    if (e == cudaSuccess) {
        h->allocs.push_back(q);
        cudaMemset(q, 0, (n ? n : 1) * sizeof(T));
    }
    *p = static_cast<T *>(q);
    return e;
}

#define MCK(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            fprintf(stderr, "lbm_mlp: %s: %s\n", #call, cudaGetErrorString(e_));  \
            return e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;    \
        }                                                                           \
    } while (0)

template <int EPI> cudaError_t gemm(lbm_mlp *h, const bf16 *A, const bf16 *Bt, int M, int N, int K, const Epi &e) {
#if LBM_MLP_MMA_SYNC
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
    k_gemm_nt<EPI><<<grid, 128, 0, h->stream>>>(A, Bt, M, N, K, e);
#else
    if (N % 32 == 0) {
        dim3 grid(N / 32, (M + TC_M - 1) / TC_M);
        k_gemm_tc<EPI, 32><<<grid, TC_THREADS, 0, h->stream>>>(A, Bt, M, N, K, e, h->err);
    } else {
        dim3 grid((N + 15) / 16, (M + TC_M - 1) / TC_M);
        k_gemm_tc<EPI, 16><<<grid, TC_THREADS, 0, h->stream>>>(A, Bt, M, N, K, e, h->err);
    }
#endif
    return cudaGetLastError();
}

cudaError_t transpose(lbm_mlp *h, const bf16 *in, bf16 *out, int R, int C) {
    dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
    k_transpose_bf16<<<grid, block, 0, h->stream>>>(in, out, R, C);
    return cudaGetLastError();
}

cudaError_t refresh(lbm_mlp *h) {
    for (int l = 0; l < h->n_layers; l++) {
        const int n = h->nout[l] * h->kpad[l];
        k_refresh_bf16<<<(n + 255) / 256, 256, 0, h->stream>>>(h->theta + h->woff[l], h->nout[l], h->nin[l],
                                                               h->kpad[l], h->Wt[l], h->W[l]);
    }
    return cudaGetLastError();
}

// forward pass from act[0] (already filled, B x 16); output in h->y
cudaError_t forward(lbm_mlp *h, int B) {
    for (int l = 0; l < h->n_layers; l++) {
        Epi e{};
        e.bias = h->theta + h->boff[l];
        if (l < h->n_layers - 1) {
            e.pre = h->pre[l];
            e.out_bf = h->act[l + 1];
            cudaError_t r = gemm<EPI_HIDDEN>(h, h->act[l], h->Wt[l], B, h->nout[l], h->kpad[l], e);
            if (r != cudaSuccess) return r;
        } else {
            e.out_f = h->y;
            cudaError_t r = gemm<EPI_OUT>(h, h->act[l], h->Wt[l], B, h->nout[l], h->kpad[l], e);
            if (r != cudaSuccess) return r;
        }
    }
    return cudaSuccess;
}

// backward pass from gf/gbf[L-1] (gradient w.r.t. the output); fills h->grad
cudaError_t backward(lbm_mlp *h, int B) {
    for (int l = h->n_layers - 1; l >= 0; l--) {
        const int N = h->nout[l], K = h->kpad[l];
        k_bias_grad<<<(N + 127) / 128, 128, 0, h->stream>>>(h->gf[l], B, N, h->grad + h->boff[l]);
        cudaError_t r = transpose(h, h->gbf[l], h->gT[l], B, N);
        if (r == cudaSuccess) r = transpose(h, h->act[l], h->actT[l], B, K);
        if (r != cudaSuccess) return r;
        Epi e{};
        e.out_f = h->dw;
        r = gemm<EPI_DW>(h, h->gT[l], h->actT[l], N, K, B, e);
        if (r != cudaSuccess) return r;
        const int cnt = N * h->nin[l];
        k_unpad<<<(cnt + 255) / 256, 256, 0, h->stream>>>(h->dw, N, K, h->nin[l], h->grad + h->woff[l]);
        if (l > 0) {
            Epi d{};
            d.out_f = h->gf[l - 1];
            d.out_bf = h->gbf[l - 1];
            d.pre_in = h->pre[l - 1];
            r = gemm<EPI_DX>(h, h->gbf[l], h->W[l], B, K, N, d);
            if (r != cudaSuccess) return r;
        }
    }
    return cudaGetLastError();
}

lbm_status load_input(lbm_mlp *h, const float *x, int B) {
    std::vector<bf16> xb((size_t)B * K0);
    for (int b = 0; b < B; b++)
        for (int j = 0; j < K0; j++) xb[(size_t)b * K0 + j] = __float2bfloat16_rn(j < h->n_in ? x[(size_t)b * h->n_in + j] : 0.f);
    MCK(cudaMemcpyAsync(h->act[0], xb.data(), xb.size() * sizeof(bf16), cudaMemcpyHostToDevice, h->stream));
    MCK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

bool bad_batch(const lbm_mlp *h, int B) { return !h || B < 16 || B % 16 || B > h->max_batch; }

// after a synchronisation: a tensor-core product that gave up waiting
lbm_status check_err(lbm_mlp *h) {
    int e = 0;
    MCK(cudaMemcpy(&e, h->err, sizeof e, cudaMemcpyDeviceToHost));
    if (e) {
        fprintf(stderr, "lbm_mlp: a tensor-core product timed out waiting for its MMAs\n");
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_mlp_create(int n_in, int hidden, int n_hidden, int n_out, int max_batch, int device, void *stream,
                          lbm_mlp **out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (n_in < 1 || n_in > K0 || hidden < 64 || hidden % 64 || n_hidden < 1 || n_out < 16 || n_out % 16 ||
        max_batch < 64 || max_batch % 64) {
        fprintf(stderr, "lbm_mlp_create: invalid shape\n");
        return LBM_ERR_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return LBM_ERR_CUDA;
    lbm_mlp *h = new lbm_mlp();
    h->device = device;
    h->n_in = n_in;
    h->n_out = n_out;
    h->hidden = hidden;
    h->n_layers = n_hidden + 1;
    h->max_batch = max_batch;
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        h->own_stream = true;
    }
    int64_t off = 0;
    int maxw = 0;
    for (int l = 0; l < h->n_layers; l++) {
        const int ni = l == 0 ? n_in : hidden, no = l == h->n_layers - 1 ? n_out : hidden;
        h->nin.push_back(ni);
        h->nout.push_back(no);
        h->kpad.push_back(l == 0 ? K0 : hidden);
        h->woff.push_back(off);
        off += (int64_t)ni * no;
        h->boff.push_back(off);
        off += no;
        maxw = std::max(maxw, no * h->kpad[l]);
    }
    h->np = off;
    bool ok = dal(h, &h->theta, off) == cudaSuccess && dal(h, &h->grad, off) == cudaSuccess &&
              dal(h, &h->m, off) == cudaSuccess && dal(h, &h->v, off) == cudaSuccess &&
              dal(h, &h->dw, maxw) == cudaSuccess && dal(h, &h->y, (size_t)max_batch * n_out) == cudaSuccess &&
              dal(h, &h->t, (size_t)max_batch * n_out) == cudaSuccess &&
              dal(h, &h->row_loss, max_batch) == cudaSuccess && dal(h, &h->idx, max_batch) == cudaSuccess &&
              dal(h, &h->err, 1) == cudaSuccess;
    h->Wt.resize(h->n_layers);
    h->W.resize(h->n_layers);
    h->act.resize(h->n_layers + 1);
    h->actT.resize(h->n_layers);
    h->pre.resize(h->n_layers);
    h->gf.resize(h->n_layers);
    h->gbf.resize(h->n_layers);
    h->gT.resize(h->n_layers);
    for (int l = 0; l < h->n_layers && ok; l++) {
        const size_t B = max_batch;
        ok = dal(h, &h->Wt[l], (size_t)h->nout[l] * h->kpad[l]) == cudaSuccess &&
             dal(h, &h->W[l], (size_t)h->nout[l] * h->kpad[l]) == cudaSuccess &&
             dal(h, &h->act[l], B * h->kpad[l]) == cudaSuccess &&
             dal(h, &h->actT[l], B * h->kpad[l]) == cudaSuccess &&
             dal(h, &h->pre[l], B * h->nout[l]) == cudaSuccess &&
             dal(h, &h->gf[l], B * h->nout[l]) == cudaSuccess &&
             dal(h, &h->gbf[l], B * h->nout[l]) == cudaSuccess &&
             dal(h, &h->gT[l], B * h->nout[l]) == cudaSuccess;
    }
    if (!ok) {
        lbm_mlp_destroy(h);
        return LBM_ERR_OOM;
    }
    *out = h;
    return LBM_OK;
}

int64_t lbm_mlp_num_params(const lbm_mlp *m) { return m ? m->np : 0; }

lbm_status lbm_mlp_set_params(lbm_mlp *h, const float *theta, int64_t n) {
    if (!h || !theta || n != h->np) return LBM_ERR_ARG;
    for (int64_t i = 0; i < n; i++)
        if (!std::isfinite(theta[i])) return LBM_ERR_ARG;
    MCK(cudaSetDevice(h->device));
    MCK(cudaMemcpyAsync(h->theta, theta, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    MCK(cudaMemsetAsync(h->m, 0, n * sizeof(float), h->stream));
    MCK(cudaMemsetAsync(h->v, 0, n * sizeof(float), h->stream));
    h->adam_steps = 0;
    MCK(refresh(h));
    MCK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_get_params(lbm_mlp *h, float *theta, int64_t n) {
    if (!h || !theta || n != h->np) return LBM_ERR_ARG;
    MCK(cudaSetDevice(h->device));
    MCK(cudaMemcpyAsync(theta, h->theta, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp *h, const float *x, int B, float *y) {
    if (bad_batch(h, B) || !x || !y) return LBM_ERR_ARG;
    MCK(cudaSetDevice(h->device));
    lbm_status s = load_input(h, x, B);
    if (s != LBM_OK) return s;
    MCK(forward(h, B));
    MCK(cudaMemcpyAsync(y, h->y, (size_t)B * h->n_out * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaStreamSynchronize(h->stream));
    return check_err(h);
}

lbm_status lbm_mlp_grad(lbm_mlp *h, const float *x, const float *dy, int B, float *g) {
    if (bad_batch(h, B) || !x || !dy || !g) return LBM_ERR_ARG;
    MCK(cudaSetDevice(h->device));
    lbm_status s = load_input(h, x, B);
    if (s != LBM_OK) return s;
    MCK(forward(h, B));
    const int L = h->n_layers - 1;
    const size_t n = (size_t)B * h->n_out;
    std::vector<bf16> db(n);
    for (size_t i = 0; i < n; i++) db[i] = __float2bfloat16_rn(dy[i]);
    MCK(cudaMemcpyAsync(h->gf[L], dy, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    MCK(cudaMemcpyAsync(h->gbf[L], db.data(), n * sizeof(bf16), cudaMemcpyHostToDevice, h->stream));
    MCK(backward(h, B));
    MCK(cudaMemcpyAsync(g, h->grad, h->np * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    MCK(cudaStreamSynchronize(h->stream));
    return check_err(h);
}

lbm_status lbm_mlp_set_data(lbm_mlp *h, const float *x, const float *t, int n) {
    if (!h || !x || !t || n < 1) return LBM_ERR_ARG;
    MCK(cudaSetDevice(h->device));
    MCK(cudaStreamSynchronize(h->stream));
    if (h->xd) cudaFree(h->xd);
    if (h->td) cudaFree(h->td);
    h->xd = h->td = nullptr;
    MCK(cudaMalloc(&h->xd, (size_t)n * h->n_in * sizeof(float)));
    MCK(cudaMalloc(&h->td, (size_t)n * h->n_out * sizeof(float)));
    MCK(cudaMemcpy(h->xd, x, (size_t)n * h->n_in * sizeof(float), cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(h->td, t, (size_t)n * h->n_out * sizeof(float), cudaMemcpyHostToDevice));
    h->n_data = n;
    return LBM_OK;
}

lbm_status lbm_mlp_train(lbm_mlp *h, const int32_t *order, int n_steps, int B, float lr, float *losses) {
    if (bad_batch(h, B) || !order || n_steps < 1 || !h->xd) return LBM_ERR_ARG;
    for (int64_t i = 0; i < (int64_t)n_steps * B; i++)
        if (order[i] < 0 || order[i] >= h->n_data) return LBM_ERR_ARG;
    MCK(cudaSetDevice(h->device));
    int32_t *ord = nullptr;
    float *dl = nullptr;
    MCK(cudaMalloc(&ord, (size_t)n_steps * B * sizeof(int32_t)));
    MCK(cudaMalloc(&dl, (size_t)n_steps * sizeof(float)));
    MCK(cudaMemcpy(ord, order, (size_t)n_steps * B * sizeof(int32_t), cudaMemcpyHostToDevice));
    const int L = h->n_layers - 1;
    const float b1 = 0.9f, b2 = 0.999f;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < n_steps && e == cudaSuccess; s++) {
        k_gather_batch<<<B, 64, 0, h->stream>>>(h->xd, h->td, ord + (size_t)s * B, B, h->n_in, h->n_out, h->act[0], h->t);
        e = forward(h, B);
        if (e != cudaSuccess) break;
        k_mse_grad<<<B, 64, 0, h->stream>>>(h->y, h->t, B, h->n_out, h->gf[L], h->gbf[L], h->row_loss);
        k_sum_loss<<<1, 256, 0, h->stream>>>(h->row_loss, B, h->n_out, dl + s);
        e = backward(h, B);
        if (e != cudaSuccess) break;
        h->adam_steps++;
        const float c1 = 1.f - powf(b1, (float)h->adam_steps), c2 = 1.f - powf(b2, (float)h->adam_steps);
        k_adam<<<(int)((h->np + 255) / 256), 256, 0, h->stream>>>(h->theta, h->grad, h->m, h->v, h->np, lr, b1, b2, c1,
                                                                    c2, 1e-8f);
        e = refresh(h);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && losses)
        e = cudaMemcpyAsync(losses, dl, (size_t)n_steps * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(ord);
    cudaFree(dl);
    MCK(e);
    return check_err(h);
}

void lbm_mlp_destroy(lbm_mlp *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void *p : h->allocs) cudaFree(p);
    if (h->xd) cudaFree(h->xd);
    if (h->td) cudaFree(h->td);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
