// Trailing update of the FP32 supernodal fronts on the 5th-generation tensor
// cores (tcgen05, TF32 inputs, FP32 accumulation in tensor memory).
//
// Section 2.3 solves the overlapping subdomain problems with direct local
// factorisations; in the mixed-precision form these factors are FP32.  The
// dense part of a front's partial Cholesky that dominates its flops is the
// symmetric rank-k update of the trailing matrix
//     F[r, c] -= sum_k P[r, k] P[c, k],   r >= c >= base,
// P the kw (<= 128) freshly factored panel columns.  Here it runs as a GEMM on
// tcgen05.mma.kind::tf32: one CTA per 128 x 128 lower tile of a front's
// trailing matrix, the panel rows of the tile's row and column ranges staged
// in shared memory in the K-major layout without swizzle (core matrices of
// 8 rows x 16 bytes), the 128 x 128 FP32 product accumulated in 128 columns
// of tensor memory, then read back with tcgen05.ld and subtracted from the
// front in global memory.  TF32 keeps 10 of FP32's 23 mantissa bits, so each
// operand is split x = hi + lo (hi = x rounded to TF32, lo = x - hi rounded to
// TF32) and the product is hi*hi + hi*lo + lo*hi ("3xTF32"): the rounding of
// lo and the dropped lo*lo term leave a relative error near 2^-22 per
// product, close to the 2^-24 of an FP32 update.
//
// Every wait on the tensor cores is bounded: if a commit does not arrive
// within the limit the kernel raises the error flag, skips the write-back,
// frees its tensor memory and returns (the host reports GL_ERR_TIMEOUT).
#include "factor.h"

namespace gl {

namespace {

constexpr int TC_M = 128, TC_N = 128;   // output tile
constexpr int TC_KC = 32;               // panel columns staged per round (4 MMAs of K = 8)
constexpr int TC_THREADS = 128;         // 4 warps: one per 32-lane quarter of tensor memory
constexpr int TC_TMEM_COLS = 128;       // FP32 accumulator columns
// one operand tile: 128 rows x 32 FP32 = 16 KB; hi and lo of A and B
constexpr int TC_TILE_BYTES = TC_M * TC_KC * 4;
constexpr int TC_SMEM = 4 * TC_TILE_BYTES + 1024;   // + alignment slack
constexpr unsigned TC_WAIT_LIMIT = 1u << 26;          // polls of an mbarrier before giving up

// Byte offset of element (row m, column k) of a 128 x 32 operand tile in the
// K-major no-swizzle layout: core matrix (m / 8, k / 4) holds 8 rows of 16 B;
// core matrices are 128 B apart along K (leading byte offset) and
// 8 x 128 B = 1024 B apart along M (stride byte offset).
constexpr uint32_t TC_LBO = 128, TC_SBO = 1024;
__device__ __forceinline__ uint32_t tile_off(int m, int k) {
    return (uint32_t)((m >> 3) * TC_SBO + (k >> 2) * TC_LBO + (m & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05 (start address, leading and
// stride byte offsets in 16-byte units, descriptor version 1 at bit 46, no
// swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(TC_LBO >> 4) << 16) |
           ((uint64_t)(TC_SBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Bounded wait for the mbarrier phase `parity`; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (unsigned it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred P1;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, P1;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float out[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) out[i] = __uint_as_float(r[i]);
}

// Stage rows [row0, row0 + 128) x panel columns [kc, kc + 32) of the front
// (column-major, leading dimension f) as hi and lo TF32 tiles; rows >= f and
// columns >= kend are zero.  Thread t stages row t.
__device__ __forceinline__ void stage_rows(const float *__restrict__ F, int f, int row0, int kc, int kend,
                                           unsigned char *hi, unsigned char *lo) {
    const int t = threadIdx.x;
    const int r = row0 + t;
#pragma unroll
    for (int k4 = 0; k4 < TC_KC; k4 += 4) {
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = kc + k4 + e;
            const float x = (r < f && k < kend) ? F[r + (int64_t)k * f] : 0.0f;
            h[e] = to_tf32(x);
            l[e] = to_tf32(x - h[e]);   // rounded, not left to the hardware's truncation
        }
        *reinterpret_cast<float4 *>(hi + tile_off(t, k4)) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(lo + tile_off(t, k4)) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

// One CTA per (front, 128 x 128 lower tile of its trailing matrix): with
// kw = min(128, p - k0) panel columns [k0, k0 + kw) and base = k0 + kw,
// F[r, c] -= sum_{k in panel} F[r, k] F[c, k] for base <= c <= r < f.
__global__ void __launch_bounds__(TC_THREADS) k_syrk_tc(const int *__restrict__ fronts,
                                                        const FrontDesc *__restrict__ D, float *__restrict__ ws,
                                                        int k0, int *__restrict__ err) {
    const FrontDesc d = D[fronts[blockIdx.x]];
    if (k0 >= d.p) return;
    const int kw = min(128, d.p - k0), f = d.p + d.q;
    const int base = k0 + kw, m = f - base;
    if (m <= 0) return;
    const int nt = (m + TC_M - 1) / TC_M;
    const int t = blockIdx.y;
    if (t >= nt * (nt + 1) / 2) return;
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int r0 = base + ti * TC_M, c0 = base + tj * TC_N;
    float *F = ws + d.front_off;

    extern __shared__ unsigned char tc_smem_raw[];
    // operand tiles on a 1024-byte boundary (16 bytes are what the descriptors need)
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *a_hi = sm, *a_lo = sm + TC_TILE_BYTES, *b_hi = sm + 2 * TC_TILE_BYTES,
                  *b_lo = sm + 3 * TC_TILE_BYTES;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ int failed;
    const int warp = threadIdx.x >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t mb = smem_addr(&mbar);

    const int kend = k0 + kw;
    uint32_t phase = 0;
    bool first = true;
    for (int kc = k0; kc < kend; kc += TC_KC) {
        stage_rows(F, f, r0, kc, kend, a_hi, a_lo);
        stage_rows(F, f, c0, kc, kend, b_hi, b_lo);
        // generic-proxy stores -> visible to the tensor cores (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_addr(a_hi), al = smem_addr(a_lo), bh = smem_addr(b_hi), bl = smem_addr(b_lo);
#pragma unroll
            for (int s = 0; s < TC_KC / 8; ++s) {
                const uint32_t ko = (uint32_t)(2 * s) * TC_LBO;    // K = 8 TF32 = two core matrices
                mma_tf32(tmem, smem_desc(ah + ko), smem_desc(bh + ko), first ? 0u : 1u);
                first = false;
                mma_tf32(tmem, smem_desc(ah + ko), smem_desc(bl + ko), 1u);
                mma_tf32(tmem, smem_desc(al + ko), smem_desc(bh + ko), 1u);
            }
            mma_commit(mb);
        }
        first = false;
        // the next round overwrites the tiles: wait until the tensor cores have read them
        if (!mbar_wait(mb, phase)) failed = 1;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (failed) break;
    }

    if (!failed) {
        // epilogue: warp w holds rows r0 + 32 w + lane; subtract the product from the front
        const int r = r0 + 32 * warp + (threadIdx.x & 31);
#pragma unroll 1
        for (int cb = 0; cb < TC_N; cb += 32) {
            float acc[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, acc);
            if (r < f) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int c = c0 + cb + j;
                    if (c < f && c <= r) F[r + (int64_t)c * f] -= acc[j];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

}  // namespace

int syrk_tc_panel() { return 128; }

void syrk_tc_level(const int *d_fronts, int n_fronts, const FrontDesc *d_fr, int k0, int max_f, float *ws,
                   int *d_err, cudaStream_t s) {
    static SmemLimit lim;
    lim.ensure(TC_SMEM, [](size_t v) {
        GL_CUDA(cudaFuncSetAttribute(k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v));
    });
    const int m = max_f - k0;   // upper bound of the trailing size over the level's fronts
    if (m <= 0) return;
    const int nt = (m + TC_M - 1) / TC_M;
    const int tiles = nt * (nt + 1) / 2;
    k_syrk_tc<<<dim3(n_fronts, tiles), TC_THREADS, TC_SMEM, s>>>(d_fronts, d_fr, ws, k0, d_err);
    GL_CUDA(cudaGetLastError());
}

}  // namespace gl
