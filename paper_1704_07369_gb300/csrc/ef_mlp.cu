// ef_mlp.cu -- the learned surrogate's multilayer perceptron: bf16 weights and activations, FP32
// accumulation, hand-written training (forward, MSE loss, backward, Adam) and inference.
//
// Layer l: pre_l = A_{l-1} W_l^T + b_l, A_l = relu(pre_l) (no activation on the last layer).
// Every product is one "TN" GEMM C[M,N] = A[M,K] B[N,K]^T with both operands K-contiguous bf16
// and an FP32 accumulator on the tensor cores: tcgen05.mma fed by TMA, with the accumulator in
// tensor memory, for the shapes it tiles (M a multiple of 128), else mma.sync m16n8k16 with 64 x 64
// tiles.  Backward products use the transposed
// copies the forward pass and the optimizer write alongside (activations^T, W^T).
// Split precision: every layer input a (the features and each hidden activation) is stored as two
// bf16 halves, hi = bf16(a) and lo = bf16(a - hi), side by side, and multiplied against the weights
// duplicated [bf16(W) | bf16(W)], so that a forward product sees a to about 16 mantissa bits while
// both tensor-core operands stay bf16.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "ef.h"
#include "ef_launch.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int BM = 64, BN = 64, BK = 32, LDS = BK + 8;   // smem row stride 40 bf16 = 80 B

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct GemmArgs {
    const bf16 *A;      // [M][lda], K contiguous
    const bf16 *B;      // [N][ldb], K contiguous
    int M, N, K, lda, ldb;
    const float *bias;  // nullable [N]
    int relu;
    float *Cf;          // nullable fp32 out [M][ldcf]  (pre-activation)
    int ldcf;
    bf16 *Cb;           // nullable bf16 out [M][ldcb]  (post-activation)
    int ldcb;
    bf16 *CbT;          // nullable bf16 transposed out [N][ldcbt]
    int ldcbt;
    int lo_off;         // > 0: also write the low halves a - bf16(a) at column / row + lo_off
    int *status;        // nullable: device status word, EF_ERR_TIMEOUT (5) when a bounded wait gives up
};

// 4 warps in 2 x 2, each 32 x 32 (2 m16 x 4 n8 tiles).  M % 64 == N % 64 == K % 32 == 0.
__global__ void __launch_bounds__(128) gemm_tn_kernel(const GemmArgs g)
{
    __shared__ __align__(16) bf16 sA[2][BM * LDS];
    __shared__ __align__(16) bf16 sB[2][BN * LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk = g.K / BK;

    auto load_tile = [&](int kt, int buf) {
        // A: 64 rows x 32 bf16 = 256 chunks of 16 B; B likewise: 2 + 2 chunks per thread
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int c = tid + i * 128;
            const int r = c >> 2, k8 = (c & 3) * 8;
            cp_async16(&sA[buf][r * LDS + k8], g.A + (size_t)(m0 + r) * g.lda + kt * BK + k8);
            cp_async16(&sB[buf][r * LDS + k8], g.B + (size_t)(n0 + r) * g.ldb + kt * BK + k8);
        }
        cp_async_commit();
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    load_tile(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            load_tile(kt + 1, buf ^ 1);
            cp_async_wait1();
        } else {
            cp_async_wait0();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm * 32 + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int c = kk + (lane >> 4) * 8;
                ldmatrix_x4(af[i], &sA[buf][r * LDS + c]);
            }
            uint32_t bfr[4][2];
#pragma unroll
            for (int j2 = 0; j2 < 2; ++j2) {      // two n8 tiles per ldmatrix.x4
                uint32_t t[4];
                const int n = wn * 32 + j2 * 16 + (lane & 7) + (lane >> 4) * 8;
                const int c = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(t, &sB[buf][n * LDS + c]);
                bfr[2 * j2][0] = t[0];
                bfr[2 * j2][1] = t[1];
                bfr[2 * j2 + 1][0] = t[2];
                bfr[2 * j2 + 1][1] = t[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j][0], bfr[j][1]);
        }
        __syncthreads();
    }
    // epilogue: c0,c1 at (row, col..col+1), c2,c3 at (row + 8, ...)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm * 32 + i * 16 + (lane >> 2) + h * 8;
                const int col = n0 + wn * 32 + j * 8 + (lane & 3) * 2;
                float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                if (g.bias) {
                    v0 += g.bias[col];
                    v1 += g.bias[col + 1];
                }
                if (g.Cf) *reinterpret_cast<float2 *>(g.Cf + (size_t)row * g.ldcf + col) = make_float2(v0, v1);
                if (g.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                const bf16 h0 = __float2bfloat16(v0), h1 = __float2bfloat16(v1);
                const bf16 l0 = __float2bfloat16(v0 - __bfloat162float(h0)), l1 = __float2bfloat16(v1 - __bfloat162float(h1));
                if (g.Cb) {
                    *reinterpret_cast<__nv_bfloat162 *>(g.Cb + (size_t)row * g.ldcb + col) = __halves2bfloat162(h0, h1);
                    if (g.lo_off)
                        *reinterpret_cast<__nv_bfloat162 *>(g.Cb + (size_t)row * g.ldcb + g.lo_off + col) =
                            __halves2bfloat162(l0, l1);
                }
                if (g.CbT) {
                    g.CbT[(size_t)col * g.ldcbt + row] = h0;
                    g.CbT[(size_t)(col + 1) * g.ldcbt + row] = h1;
                    if (g.lo_off) {
                        g.CbT[(size_t)(g.lo_off + col) * g.ldcbt + row] = l0;
                        g.CbT[(size_t)(g.lo_off + col + 1) * g.ldcbt + row] = l1;
                    }
                }
            }
}

// ------------------------------------------------------------ tcgen05 GEMM ---------------
// The same product and epilogue on the 5th-generation tensor cores: one CTA of 4 warps per
// 128 x TN tile of C, K in blocks of 64.  Thread 0 runs the pipeline: TMA loads (128-byte
// swizzle) of the A and B tiles of a K block into one of TC_STAGES shared-memory stages, each
// stage with a "full" mbarrier (TMA bytes arrived) and an "empty" one (its MMAs done, committed by
// tcgen05.commit); tcgen05.mma kind::f16 (M = 128, N = TN, K = 16) accumulates in tensor memory;
// a stage is refilled once the MMAs that read it are complete, after the next block's MMAs have
// been queued.  The epilogue reads the accumulator with tcgen05.ld (warp w owns tensor-memory
// lanes, i.e. rows, 32w .. 32w+31).  Every mbarrier wait is bounded.  A wait that gives up stops
// the pipeline, records EF_ERR_TIMEOUT in the status word, waits (bounded) for the CTA's copies
// and MMAs still in flight, and writes NaN for the tile without reading the accumulator; the
// tensor memory is released in every case.
constexpr int TC_BM = 128, TC_BK = 64, TC_STAGES = 4;

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr)
{
    // K-major operand with 128-byte swizzle: start address, leading offset unused (1), stride 1024
    // bytes between 8-row groups, descriptor version 1, layout type 2 (128-byte swizzle)
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}

// instruction descriptor, kind::f16: FP32 accumulator, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Bounded wait on one mbarrier phase: gives up after about one second of device time (or 2^26
// polls), far beyond any wait of a healthy pipeline (microseconds).
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int it = 0; it < (1 << 26); ++it) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 1023) == 1023) {
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 1000000000ull) return false;
        }
    }
    return false;
}

template <int TN>
__global__ void __launch_bounds__(128, 1) gemm_tc_kernel(const __grid_constant__ CUtensorMap tA,
                                                         const __grid_constant__ CUtensorMap tB, const GemmArgs g)
{
    constexpr int A_BYTES = TC_BM * TC_BK * 2, B_BYTES = TN * TC_BK * 2, STAGE = A_BYTES + B_BYTES;
    constexpr int TCOLS = TN <= 64 ? 64 : (TN <= 128 ? 128 : 256);     // tensor-memory columns
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char *tc_smem = (unsigned char *)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);   // swizzle atoms
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TN;
    const int nk = g.K / TC_BK;
    const uint32_t sbase = smem_u32(tc_smem);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tA));
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(&tB));
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = tmem_base;

    __shared__ int s_ok;
    if (tid == 0) {
        // pend[st]: a TMA load into stage st was issued and its "full" phase not yet waited for;
        // ncommit[st]: commits of MMAs reading stage st.  Each stage has at most one outstanding
        // phase of either barrier (a stage is refilled only after both were waited for), so every
        // parity below names one phase.
        bool ok = true;
        bool pend[TC_STAGES];
        uint32_t fph[TC_STAGES], eph[TC_STAGES];
        int ncommit[TC_STAGES];
        int kb_last = -1;                                // the last K block whose MMAs were committed
        auto issue = [&](int kb, int st) {
            const uint32_t a0 = sbase + st * STAGE, b0 = a0 + A_BYTES, bar = smem_u32(&full[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(STAGE));
            asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
                         ::"r"(a0), "l"(&tA), "r"(kb * TC_BK), "r"(m0), "r"(bar) : "memory");
            asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
                         ::"r"(b0), "l"(&tB), "r"(kb * TC_BK), "r"(n0), "r"(bar) : "memory");
            pend[st] = true;
        };
        for (int i = 0; i < TC_STAGES; ++i) {
            fph[i] = eph[i] = 0;
            pend[i] = false;
            ncommit[i] = 0;
            if (i < nk) issue(i, i);
        }
        for (int kb = 0; kb < nk; ++kb) {
            const int st = kb % TC_STAGES;
            if (!tc_wait(smem_u32(&full[st]), fph[st])) { ok = false; break; }
            pend[st] = false;
            fph[st] ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
            const uint32_t a0 = sbase + st * STAGE, b0 = a0 + A_BYTES;
#pragma unroll
            for (int k16 = 0; k16 < TC_BK / 16; ++k16) {
                const uint64_t ad = tc_sdesc(a0 + k16 * 32), bd = tc_sdesc(b0 + k16 * 32);
                const uint32_t acc = (kb > 0 || k16 > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(tmem), "l"(ad), "l"(bd), "r"(tc_idesc(TC_BM, TN)), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         ::"r"(smem_u32(&empty[st])));
            ++ncommit[st];
            kb_last = kb;
            const int nxt = kb - 1 + TC_STAGES;          // refill the stage of kb - 1
            if (kb >= 1 && nxt < nk) {
                const int pb = (kb - 1) % TC_STAGES;
                if (!tc_wait(smem_u32(&empty[pb]), eph[pb])) { ok = false; break; }
                eph[pb] ^= 1;
                issue(nxt, pb);
            }
        }
        // the last commit covers every MMA issued before it (tcgen05.commit tracks all prior
        // asynchronous tcgen05 operations of this thread)
        const int L = kb_last >= 0 ? kb_last % TC_STAGES : 0;
        if (ok && kb_last >= 0) ok = tc_wait(smem_u32(&empty[L]), (uint32_t)((ncommit[L] - 1) & 1));
        if (!ok) {
            // a wait gave up: record it, then wait (again bounded) for this CTA's own copies and
            // MMAs still in flight before the accumulator is released and the CTA exits
            if (g.status) atomicCAS(g.status, 0, 5);     // EF_ERR_TIMEOUT
            for (int i = 0; i < TC_STAGES; ++i)
                if (pend[i]) tc_wait(smem_u32(&full[i]), fph[i]);
            if (kb_last >= 0) tc_wait(smem_u32(&empty[L]), (uint32_t)((ncommit[L] - 1) & 1));
        }
        s_ok = ok ? 1 : 0;
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const bool ok = s_ok != 0;

    const int row = m0 + warp * 32 + lane;
    const float bad = __int_as_float(0x7fc00000);
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 8) {
        uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (ok) {            // CTA-uniform: after a give-up the accumulator is not read
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
        }
        const int col = n0 + c0;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            v[j] = ok ? __uint_as_float(r[j]) : bad;
            if (g.bias) v[j] += g.bias[col + j];
        }
        if (g.Cf) {
            float4 *d = reinterpret_cast<float4 *>(g.Cf + (size_t)row * g.ldcf + col);
            d[0] = make_float4(v[0], v[1], v[2], v[3]);
            d[1] = make_float4(v[4], v[5], v[6], v[7]);
        }
        if (g.relu) {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = fmaxf(v[j], 0.f);
        }
        bf16 hi[8], lo[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            hi[j] = __float2bfloat16(v[j]);
            lo[j] = __float2bfloat16(v[j] - __bfloat162float(hi[j]));
        }
        if (g.Cb) {
            *reinterpret_cast<uint4 *>(g.Cb + (size_t)row * g.ldcb + col) = *reinterpret_cast<const uint4 *>(hi);
            if (g.lo_off)
                *reinterpret_cast<uint4 *>(g.Cb + (size_t)row * g.ldcb + g.lo_off + col) = *reinterpret_cast<const uint4 *>(lo);
        }
        if (g.CbT) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                g.CbT[(size_t)(col + j) * g.ldcbt + row] = hi[j];
                if (g.lo_off) g.CbT[(size_t)(g.lo_off + col + j) * g.ldcbt + row] = lo[j];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TCOLS));
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the driver)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// rows x K bf16 operand with row stride ld elements, boxes of 64 K-elements x box_rows rows
bool tile_map(CUtensorMap *m, const bf16 *base, int rows, int K, int ld, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (uintptr_t)base % 16) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int TN>
cudaError_t gemm_tc(const GemmArgs &g, bool *used, cudaStream_t s)
{
    constexpr size_t smem = (size_t)TC_STAGES * (TC_BM * TC_BK * 2 + TN * TC_BK * 2) + 1024;
    *used = false;
    CUtensorMap tA, tB;
    if (!tile_map(&tA, g.A, g.M, g.K, g.lda, TC_BM) || !tile_map(&tB, g.B, g.N, g.K, g.ldb, TN)) return cudaSuccess;
    static unsigned long long set_on = 0;    // devices on which the attribute has been raised
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(__atomic_load_n(&set_on, __ATOMIC_ACQUIRE) & bit)) {
        e = cudaFuncSetAttribute(gemm_tc_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        __atomic_fetch_or(&set_on, bit, __ATOMIC_ACQ_REL);
    }
    dim3 grid(g.N / TN, g.M / TC_BM);
    gemm_tc_kernel<TN><<<grid, 128, smem, s>>>(tA, tB, g);
    *used = true;
    return cudaGetLastError();
}

// tcgen05 for the shapes it tiles (M multiple of 128, K of 64, N of 64, 16-byte aligned rows) with at
// least one tile per SM, the mma.sync kernel for the rest (and wherever a tensor map cannot be made)
cudaError_t gemm(const GemmArgs &g, cudaStream_t s)
{
    const bool aligned = g.lda % 8 == 0 && g.ldb % 8 == 0 && (!g.Cf || g.ldcf % 4 == 0) && (!g.Cb || g.ldcb % 8 == 0) &&
                         g.lo_off % 8 == 0;
    if (g.M % TC_BM == 0 && g.K % TC_BK == 0 && aligned) {
        // the widest N tile that still gives every SM a tile; small products (the training batch)
        // keep the 64 x 64 kernel, whose many CTAs fill the device
        static int sms = 0;
        if (!sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (sms <= 0) sms = 1;
        }
        const int64_t mt = g.M / TC_BM;
        auto fills = [&](int tn) { return g.N % tn == 0 && mt * (g.N / tn) >= sms; };
        bool used = false;
        cudaError_t e = cudaSuccess;
        if (fills(256)) e = gemm_tc<256>(g, &used, s);
        else if (fills(192)) e = gemm_tc<192>(g, &used, s);
        else if (fills(128)) e = gemm_tc<128>(g, &used, s);
        else if (fills(64)) e = gemm_tc<64>(g, &used, s);
        if (e != cudaSuccess || used) return e;
    }
    if (g.M % BM || g.N % BN || g.K % BK) return cudaErrorInvalidValue;
    dim3 grid(g.N / BN, g.M / BM);
    gemm_tn_kernel<<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

// X (fp32 [B][ldx], first nin used) -> split bf16 [B][2 ninp] (hi | lo) and its transpose
// [2 ninp][B]; pad zeroed.
__global__ void pack_input_kernel(const float *X, int ldx, int nin, int ninp, int64_t B, bf16 *Xb, bf16 *XbT)
{
    const int64_t total = B * ninp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / ninp;
        const int j = (int)(i % ninp);
        const float v = j < nin ? X[b * ldx + j] : 0.f;
        const bf16 h = __float2bfloat16(v);
        const bf16 l = __float2bfloat16(v - __bfloat162float(h));
        Xb[b * 2 * ninp + j] = h;
        Xb[b * 2 * ninp + ninp + j] = l;
        if (XbT) {
            XbT[(size_t)j * B + b] = h;
            XbT[(size_t)(ninp + j) * B + b] = l;
        }
    }
}

// g[o][k] = dW2[o][k] + dW2[o][in + k]: the weight gradient of the tied hi / lo halves
__global__ void fold_split_kernel(const float *dW2, int out, int in, float *g)
{
    const int64_t n = (int64_t)out * in;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i / in), k = (int)(i % in);
        g[i] = dW2[(size_t)o * 2 * in + k] + dW2[(size_t)o * 2 * in + in + k];
    }
}

// MSE loss over the first nout outputs (optionally weighted): loss = sum w_j (y - t)^2 / (B n_w),
// dY = 2 w_j (y - t) / (B n_w) in bf16 [B][noutp] and [noutp][B] (pad rows zero).
__global__ void mse_kernel(const float *Y, int ldy_pred, const float *T, int ldt, const float *wmask, const float *roww,
                           int nout, int noutp, int64_t B, float inv_count, bf16 *dY, bf16 *dYT, float *loss)
{
    float acc = 0.f;
    const int64_t total = B * noutp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / noutp;
        const int j = (int)(i % noutp);
        float g = 0.f;
        if (j < nout) {
            const float w = (wmask ? wmask[j] : 1.f) * (roww ? roww[b] : 1.f);
            const float d = Y[b * ldy_pred + j] - T[b * ldt + j];
            acc += w * d * d;
            g = 2.f * w * d * inv_count;
        }
        const bf16 h = __float2bfloat16(g);
        dY[i] = h;
        dYT[(size_t)j * B + b] = h;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(loss, t * inv_count);
    }
}

// dPre = dA * (pre > 0), as bf16 [B][n] and [n][B]
__global__ void relu_back_kernel(const float *dA, const float *pre, int64_t B, int n, bf16 *dP, bf16 *dPT)
{
    const int64_t total = B * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / n;
        const int j = (int)(i % n);
        const float g = pre[i] > 0.f ? dA[i] : 0.f;
        const bf16 h = __float2bfloat16(g);
        dP[i] = h;
        dPT[(size_t)j * B + b] = h;
    }
}

// db[j] = sum_b dYT[j][b]
__global__ void rowsum_kernel(const bf16 *dYT, int64_t B, int n, float *db)
{
    const int j = blockIdx.x;
    if (j >= n) return;
    float acc = 0.f;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) acc += __bfloat162float(dYT[(size_t)j * B + b]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        db[j] = t;
    }
}

// Adam on a parameter block (fp32 master p), then the bf16 copies W[out][in] and W^T[in][out].
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2, int out, int in, bf16 *Wb, bf16 *WbT)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (Wb) {
            const int o = (int)(i / in), k = (int)(i % in);
            const bf16 h = __float2bfloat16(pi);
            Wb[(size_t)o * 2 * in + k] = h;
            Wb[(size_t)o * 2 * in + in + k] = h;
            WbT[(size_t)k * out + o] = h;
        }
    }
}

__global__ void refresh_bf16_kernel(const float *p, int out, int in, bf16 *Wb, bf16 *WbT)
{
    const int64_t n = (int64_t)out * in;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(i / in), k = (int)(i % in);
        const bf16 h = __float2bfloat16(p[i]);
        Wb[(size_t)o * 2 * in + k] = h;
        Wb[(size_t)o * 2 * in + in + k] = h;
        WbT[(size_t)k * out + o] = h;
    }
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

int pad64(int x) { return (x + 63) / 64 * 64; }

}  // namespace

// ------------------------------------------------------------------ MLP object --------------

struct ef_mlp_s {
    int nin, nh, nl, nout;          // nl = number of weight layers (>= 2)
    int ninp, noutp;                // padded to 64
    int64_t max_batch;
    std::vector<int> din, dout;     // padded fan-in / fan-out per layer
    std::vector<int64_t> woff, boff;
    int64_t nparams = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;     // fp32 master, grad, Adam
    std::vector<bf16 *> Wb, WbT;    // per layer [out][in], [in][out]
    // activations for max_batch
    bf16 *Xb = nullptr, *XbT = nullptr;
    std::vector<float *> pre;       // [B][out_l]
    std::vector<bf16 *> act, actT;  // [B][out_l], [out_l][B] (hidden layers)
    float *dA = nullptr;            // [B][max out] fp32
    float *dW2 = nullptr;           // [max out][2 max in] fp32: gradient of the split halves
    bf16 *dY = nullptr, *dYT = nullptr;
    int64_t step = 0;
    int device = 0;
    int *status = nullptr;          // device status word (EF_ERR_TIMEOUT from a GEMM's bounded waits)
    int h_status = 0;
};

namespace {

ef_status mlp_fail(ef_status s, const std::string &m)
{
    ef::set_last_error(m.c_str());
    return s;
}

ef_status cuda_err(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    ef::set_last_error(m.c_str());
    return e == cudaErrorMemoryAllocation ? EF_ERR_OOM : EF_ERR_CUDA;
}

void mlp_free(ef_mlp_s *n)
{
    if (!n) return;
    cudaFree(n->p);
    cudaFree(n->g);
    cudaFree(n->m);
    cudaFree(n->v);
    for (auto q : n->Wb) cudaFree(q);
    for (auto q : n->WbT) cudaFree(q);
    cudaFree(n->Xb);
    cudaFree(n->XbT);
    for (auto q : n->pre) cudaFree(q);
    for (auto q : n->act) cudaFree(q);
    for (auto q : n->actT) cudaFree(q);
    cudaFree(n->dA);
    cudaFree(n->dW2);
    cudaFree(n->dY);
    cudaFree(n->dYT);
    cudaFree(n->status);
    delete n;
}

// forward pass for batch B (multiple of 64) from the packed input n->Xb
ef_status mlp_forward_packed(ef_mlp_s *n, int64_t B, float *Yout, int ldy, bool keep_T, cudaStream_t s)
{
    for (int l = 0; l < n->nl; ++l) {
        GemmArgs g{};
        g.A = l == 0 ? n->Xb : n->act[l - 1];
        g.lda = 2 * n->din[l];
        g.B = n->Wb[l];
        g.ldb = 2 * n->din[l];
        g.M = (int)B;
        g.N = n->dout[l];
        g.K = 2 * n->din[l];
        g.bias = n->p + n->boff[l];
        const bool last = l + 1 == n->nl;
        g.relu = last ? 0 : 1;
        g.Cf = last ? Yout : n->pre[l];
        g.ldcf = last ? ldy : n->dout[l];
        g.Cb = last ? nullptr : n->act[l];
        g.ldcb = 2 * n->dout[l];
        g.CbT = (last || !keep_T) ? nullptr : n->actT[l];
        g.ldcbt = (int)B;
        g.lo_off = n->dout[l];
        g.status = n->status;
        cudaError_t e = gemm(g, s);
        if (e != cudaSuccess) return cuda_err(e, "mlp gemm");
    }
    return EF_OK;
}

}  // namespace

extern "C" {

ef_status ef_mlp_create(int nin, int nhidden, int nlayers, int nout, int64_t max_batch, uint64_t seed, ef_mlp_t *out)
{
    if (!out) return mlp_fail(EF_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (nin < 1 || nhidden < 1 || nout < 1 || nlayers < 2 || max_batch < 64 || max_batch % 64)
        return mlp_fail(EF_ERR_INVALID_ARG, "need nin, nhidden, nout >= 1, nlayers >= 2, max_batch a positive multiple of 64");
    ef_mlp_s *n = new ef_mlp_s();
    n->nin = nin;
    n->nh = nhidden;
    n->nl = nlayers;
    n->nout = nout;
    n->ninp = pad64(nin);
    n->noutp = pad64(nout);
    n->max_batch = max_batch;
    cudaGetDevice(&n->device);
    const int nhp = pad64(nhidden);
    for (int l = 0; l < nlayers; ++l) {
        n->din.push_back(l == 0 ? n->ninp : nhp);
        n->dout.push_back(l + 1 == nlayers ? n->noutp : nhp);
    }
    for (int l = 0; l < nlayers; ++l) {
        n->woff.push_back(n->nparams);
        n->nparams += (int64_t)n->dout[l] * n->din[l];
        n->boff.push_back(n->nparams);
        n->nparams += n->dout[l];
    }
    // He-normal initialisation of the real (unpadded) weights, zero biases and padding
    std::vector<float> h((size_t)n->nparams, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < nlayers; ++l) {
        const int fin = l == 0 ? nin : nhidden, fout = l + 1 == nlayers ? nout : nhidden;
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / fin) * (l + 1 == nlayers ? 0.5 : 1.0));
        for (int o = 0; o < fout; ++o)
            for (int k = 0; k < fin; ++k) h[(size_t)(n->woff[l] + (int64_t)o * n->din[l] + k)] = (float)nd(rng);
    }
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
        if (e == cudaSuccess) e = cudaMemset(*ptr, 0, bytes);
    };
    alloc((void **)&n->p, n->nparams * 4);
    alloc((void **)&n->g, n->nparams * 4);
    alloc((void **)&n->m, n->nparams * 4);
    alloc((void **)&n->v, n->nparams * 4);
    if (e == cudaSuccess) e = cudaMemcpy(n->p, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
    n->Wb.assign(nlayers, nullptr);
    n->WbT.assign(nlayers, nullptr);
    n->pre.assign(nlayers, nullptr);
    n->act.assign(nlayers, nullptr);
    n->actT.assign(nlayers, nullptr);
    int maxd = 0;
    for (int l = 0; l < nlayers; ++l) {
        alloc((void **)&n->Wb[l], (size_t)n->dout[l] * 2 * n->din[l] * 2);
        alloc((void **)&n->WbT[l], (size_t)n->dout[l] * n->din[l] * 2);
        alloc((void **)&n->pre[l], (size_t)max_batch * n->dout[l] * 4);
        alloc((void **)&n->act[l], (size_t)max_batch * 2 * n->dout[l] * 2);
        alloc((void **)&n->actT[l], (size_t)max_batch * 2 * n->dout[l] * 2);
        maxd = std::max(maxd, std::max(n->dout[l], n->din[l]));
    }
    alloc((void **)&n->Xb, (size_t)max_batch * 2 * n->ninp * 2);
    alloc((void **)&n->XbT, (size_t)max_batch * 2 * n->ninp * 2);
    alloc((void **)&n->dW2, (size_t)maxd * 2 * maxd * 4);
    alloc((void **)&n->dA, (size_t)max_batch * maxd * 4);
    alloc((void **)&n->dY, (size_t)max_batch * maxd * 2);
    alloc((void **)&n->dYT, (size_t)max_batch * maxd * 2);
    alloc((void **)&n->status, sizeof(int));
    if (e != cudaSuccess) {
        mlp_free(n);
        return cuda_err(e, "mlp allocation");
    }
    for (int l = 0; l < nlayers; ++l) {
        refresh_bf16_kernel<<<grid_for((int64_t)n->dout[l] * n->din[l]), 256>>>(n->p + n->woff[l], n->dout[l], n->din[l],
                                                                                n->Wb[l], n->WbT[l]);
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        mlp_free(n);
        return cuda_err(e, "mlp init");
    }
    *out = n;
    return EF_OK;
}

ef_status ef_mlp_destroy(ef_mlp_t n)
{
    if (!n) return mlp_fail(EF_ERR_INVALID_ARG, "null mlp");
    mlp_free(n);
    return EF_OK;
}

ef_status ef_mlp_status(ef_mlp_t n, int sync, int reset)
{
    if (!n) return mlp_fail(EF_ERR_INVALID_ARG, "null mlp");
    if (sync) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_err(e, "device synchronize");
        e = cudaMemcpy(&n->h_status, n->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_err(e, "status read");
        if (reset) {
            e = cudaMemset(n->status, 0, sizeof(int));
            if (e != cudaSuccess) return cuda_err(e, "status reset");
        }
    }
    const int st = n->h_status;
    if (reset) n->h_status = 0;
    return (ef_status)st;
}

ef_status ef_mlp_info(ef_mlp_t n, int64_t info[8])
{
    if (!n || !info) return mlp_fail(EF_ERR_INVALID_ARG, "null mlp or info");
    info[0] = n->nin;
    info[1] = n->nh;
    info[2] = n->nl;
    info[3] = n->nout;
    info[4] = n->nparams;
    info[5] = n->ninp;
    info[6] = n->noutp;
    info[7] = n->max_batch;
    return EF_OK;
}

ef_status ef_mlp_params(ef_mlp_t n, float *host, int set)
{
    if (!n || !host) return mlp_fail(EF_ERR_INVALID_ARG, "null mlp or buffer");
    cudaError_t e = set ? cudaMemcpy(n->p, host, n->nparams * 4, cudaMemcpyHostToDevice)
                        : cudaMemcpy(host, n->p, n->nparams * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "mlp params");
    if (set) {
        for (int l = 0; l < n->nl; ++l)
            refresh_bf16_kernel<<<grid_for((int64_t)n->dout[l] * n->din[l]), 256>>>(n->p + n->woff[l], n->dout[l],
                                                                                    n->din[l], n->Wb[l], n->WbT[l]);
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_err(e, "mlp params");
    }
    return EF_OK;
}

ef_status ef_mlp_forward(ef_mlp_t n, const float *X, int ldx, float *Y, int ldy, int64_t B, ef_stream_t stream)
{
    if (!n || !X || !Y) return mlp_fail(EF_ERR_INVALID_ARG, "null mlp, X or Y");
    if (B < 0 || B % 64 || B > n->max_batch) return mlp_fail(EF_ERR_INVALID_ARG, "batch must be a multiple of 64 <= max_batch");
    if (ldx < n->nin || ldy < n->noutp || ldy % 2) return mlp_fail(EF_ERR_INVALID_ARG, "ldx >= nin, ldy >= padded nout (even)");
    if (B == 0) return EF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    pack_input_kernel<<<grid_for(B * n->ninp), 256, 0, s>>>(X, ldx, n->nin, n->ninp, B, n->Xb, nullptr);
    return mlp_forward_packed(n, B, Y, ldy, false, s);
}

// loss and gradients (into the MLP's gradient buffer); optionally the Adam update
static ef_status mlp_grad_impl(ef_mlp_s *n, const float *X, int ldx, const float *T, int ldt, const float *wmask,
                               const float *roww, int64_t B, float *loss_dev, cudaStream_t s)
{
    pack_input_kernel<<<grid_for(B * n->ninp), 256, 0, s>>>(X, ldx, n->nin, n->ninp, B, n->Xb, n->XbT);
    // forward (last layer's fp32 output into dA as scratch)
    ef_status st = mlp_forward_packed(n, B, n->dA, n->noutp, true, s);
    if (st != EF_OK) return st;
    // weighted count for the mean
    float nw = (float)n->nout;
    (void)nw;
    cudaError_t e = cudaMemsetAsync(loss_dev, 0, sizeof(float), s);
    if (e != cudaSuccess) return cuda_err(e, "loss reset");
    mse_kernel<<<grid_for(B * n->noutp), 256, 0, s>>>(n->dA, n->noutp, T, ldt, wmask, roww, n->nout, n->noutp, B,
                                                       1.f / ((float)B * (float)n->nout), n->dY, n->dYT, loss_dev);
    // backward
    for (int l = n->nl - 1; l >= 0; --l) {
        const int out = n->dout[l], in = n->din[l];
        // dW_l = dPre_l^T A_{l-1}:  M = out, N = in, K = B; A = dPreT [out][B], B = A_{l-1}^T [in][B]
        GemmArgs g{};
        g.A = n->dYT;
        g.lda = (int)B;
        g.B = l == 0 ? n->XbT : n->actT[l - 1];
        g.ldb = (int)B;
        g.M = out;
        g.N = 2 * in;
        g.K = (int)B;
        g.Cf = n->dW2;
        g.ldcf = 2 * in;
        g.status = n->status;
        e = gemm(g, s);
        if (e != cudaSuccess) return cuda_err(e, "mlp grad gemm");
        fold_split_kernel<<<grid_for((int64_t)out * in), 256, 0, s>>>(n->dW2, out, in, n->g + n->woff[l]);
        rowsum_kernel<<<out, 256, 0, s>>>(n->dYT, B, out, n->g + n->boff[l]);
        if (l == 0) break;
        // dA_{l-1} = dPre_l W_l:  M = B, N = in, K = out; A = dPre [B][out], B = W^T [in][out]
        GemmArgs h{};
        h.A = n->dY;
        h.lda = out;
        h.B = n->WbT[l];
        h.ldb = out;
        h.M = (int)B;
        h.N = in;
        h.K = out;
        h.Cf = n->dA;
        h.ldcf = in;
        h.status = n->status;
        e = gemm(h, s);
        if (e != cudaSuccess) return cuda_err(e, "mlp backprop gemm");
        relu_back_kernel<<<grid_for(B * in), 256, 0, s>>>(n->dA, n->pre[l - 1], B, in, n->dY, n->dYT);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "mlp backward");
    return EF_OK;
}

ef_status ef_mlp_grad(ef_mlp_t n, const float *X, int ldx, const float *T, int ldt, const float *wmask,
                      const float *rowweight, int64_t B, float *loss_dev, float *grad_dev, ef_stream_t stream)
{
    if (!n || !X || !T || !loss_dev) return mlp_fail(EF_ERR_INVALID_ARG, "null argument");
    if (B <= 0 || B % 64 || B > n->max_batch) return mlp_fail(EF_ERR_INVALID_ARG, "batch must be a multiple of 64 <= max_batch");
    if (ldx < n->nin || ldt < n->nout) return mlp_fail(EF_ERR_INVALID_ARG, "ldx >= nin, ldt >= nout");
    cudaStream_t s = (cudaStream_t)stream;
    ef_status st = mlp_grad_impl(n, X, ldx, T, ldt, wmask, rowweight, B, loss_dev, s);
    if (st != EF_OK) return st;
    if (grad_dev) {
        cudaError_t e = cudaMemcpyAsync(grad_dev, n->g, n->nparams * 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_err(e, "grad copy");
    }
    return EF_OK;
}

ef_status ef_mlp_train_step(ef_mlp_t n, const float *X, int ldx, const float *T, int ldt, const float *wmask,
                            const float *rowweight, int64_t B, float lr, float *loss_dev, ef_stream_t stream)
{
    ef_status st = ef_mlp_grad(n, X, ldx, T, ldt, wmask, rowweight, B, loss_dev, nullptr, stream);
    if (st != EF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
    for (int l = 0; l < n->nl; ++l) {
        const int64_t nw = (int64_t)n->dout[l] * n->din[l];
        adam_kernel<<<grid_for(nw), 256, 0, s>>>(n->p + n->woff[l], n->g + n->woff[l], n->m + n->woff[l],
                                                 n->v + n->woff[l], nw, lr, b1, b2, eps, c1, c2, n->dout[l], n->din[l],
                                                 n->Wb[l], n->WbT[l]);
        adam_kernel<<<grid_for(n->dout[l]), 256, 0, s>>>(n->p + n->boff[l], n->g + n->boff[l], n->m + n->boff[l],
                                                         n->v + n->boff[l], n->dout[l], lr, b1, b2, eps, c1, c2, 0, 1,
                                                         nullptr, nullptr);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "adam");
    return EF_OK;
}

}  // extern "C"
