// Reverse-mode adjoint accumulation of TF32 instances (states padded to 64)
// on the 5th-generation tensor cores: tcgen05.mma kind::tf32 with TMEM
// accumulators.
//
// For a parent n with children a, b, a category r and a pattern p the two
// contractions are (Sec. "Algorithmic advances": pre-order partials; the
// likelihood is linear in each child's transition matrix)
//   v_c[p] = P_c,r x_c[p]                                   (states i)
//   U_a[p] = (w_p / L_p) w_r q_n[p] o v_b[p],  U_b likewise with v_a
//   M_c,r += sum_p U_c[p] x_c[p]^T                          (64 x 64)
// A block takes one (parent, category, chunk of patterns), tiles of 128
// patterns, four epilogue warps (thread = pattern = TMEM lane) and one
// issuing warp.
//
// First product: A = x_c from tensor memory (each thread stores its own
// pattern's row; with split partials also x_lo), B = P_c hi and lo
// (K-major, 128-byte swizzle, resident for the whole chunk): v_c = x P_hi^T
// + x P_lo^T (+ x_lo P_hi^T), M = 128 patterns, N = 64, K = 64.
//
// Second product: the contraction runs over patterns, and a tf32 operand
// must be K-major (its 32-bit elements contiguous along K), so each warp
// writes its 32 patterns transposed: the A operand stacks U_hi^T (rows
// 0-63) over U_lo^T (rows 64-127), one M = 128 operand, and B is x_c^T
// (x_hi^T, with split partials also x_lo^T). The accumulator then holds
// U_hi^T x and U_lo^T x in lanes 0-63 and 64-127, added when the chunk
// ends; one M = 128 instruction per K step carries both halves of the
// split. Each warp owns its transposed slice (32 patterns = one 128-byte
// K chunk), so the four warps write in parallel and the issuing thread
// consumes the slices in a fixed order.
//
// Products are accumulated in FP32 over at most 4,096 patterns per chunk
// and written as FP64 per-chunk partial sums, like the other accumulation
// kernels. Every wait is bounded (elapsed time and a shared abort flag);
// a wait that gives up sets a flag the host reports as TL_ERR_TIMEOUT.
#include <cuda.h>

#include "tl_internal.cuh"
#include "tl_tcgen05.cuh"

namespace tl {
namespace {
using namespace tc5;

constexpr int kAdjEpiWarps = 4;
constexpr int kAdjThreads = 32 * (kAdjEpiWarps + 1);
constexpr int kMatBytes = 64 * 128;             // one K chunk (32 states) of a 64-row matrix
constexpr int kPBytes = 2 * kMatBytes;          // a 64 x 64 matrix: two K chunks, 16 KB
constexpr int kStackBytes = 128 * 128;          // A of the second product: 128 rows x 32 patterns
// TMEM columns: x_c, v_c, M_c and x_lo,c (split partials) for c = a, b
constexpr uint32_t kColX = 0, kColV = 128, kColM = 256, kColXL = 384;
constexpr int kAdjTmemCols = 512;

template <bool SPLITX>
struct AdjTcLayout {
    // per warp: stacked U^T, x_hi^T (and x_lo^T)
    static constexpr int slice = kStackBytes + (SPLITX ? 2 : 1) * kMatBytes;
    static constexpr int p_area = 4 * kPBytes;      // P_a hi, P_a lo, P_b hi, P_b lo
    static constexpr size_t bytes = (size_t)p_area + (size_t)kAdjEpiWarps * slice;
    static constexpr size_t smem = bytes + 1024;    // room to align the base to 1024
};

// Byte offset of element (row, k) in a K-major, 128-byte-swizzled operand
// chunk (rows of 32 values; the 16-byte unit j of row r sits at j ^ (r & 7)).
__device__ __forceinline__ uint32_t sw_off(int row, int k) {
    return (uint32_t)(row * 128 + ((((k >> 2) ^ (row & 7)) & 7) << 4) + (k & 3) * 4);
}
__device__ __forceinline__ void sts(unsigned char* base, uint32_t off, float v) {
    *reinterpret_cast<float*>(base + off) = v;
}
// A 64-float row of global memory (16-byte aligned).
__device__ __forceinline__ void load_row(const float* src, float* v) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4 f[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) f[u] = s4[u];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        v[4 * u] = f[u].x;
        v[4 * u + 1] = f[u].y;
        v[4 * u + 2] = f[u].z;
        v[4 * u + 3] = f[u].w;
    }
}

template <bool SPLITX>
__global__ void __launch_bounds__(kAdjThreads, 1)
k_adj_tc(const AdjOp<float>* __restrict__ ops, AdjArgs a, double* __restrict__ mpart) {
    using L = AdjTcLayout<SPLITX>;
    extern __shared__ __align__(1024) unsigned char smem_adj[];
    unsigned char* parea = smem_adj + ((1024u - (smem_u32(smem_adj) & 1023u)) & 1023u);
    unsigned char* slices = parea + L::p_area;
    __shared__ __align__(8) uint64_t a_ready, v_full, s_full[kAdjEpiWarps], s_empty[kAdjEpiWarps],
        done;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;  // bit 0 a_ready, 1 s_full, 2 v_full, 3 s_empty, 4 done
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_v = &abort_sh;
    const AdjOp<float>& op = ops[blockIdx.x];
    const int r = blockIdx.y, S = a.S;
    const int p_begin = blockIdx.z * a.chunk;
    const int p_end = min(a.Ppad, p_begin + a.chunk);
    const int n_tiles = p_end > p_begin ? (p_end - p_begin) / kTcM : 0;

    if (tid == 0) {
        abort_sh = 0;
        mbar_init(&a_ready, kAdjEpiWarps);
        mbar_init(&v_full, 1);
        for (int w = 0; w < kAdjEpiWarps; ++w) {
            mbar_init(&s_full[w], 1);
            mbar_init(&s_empty[w], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == kAdjEpiWarps) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                smem_u32(&tmem_sh)),
            "r"(kAdjTmemCols)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    // B operands of the first product: P_c[i][j] split as TF32 hi + lo,
    // row i (output state), K = j
    for (int idx = tid; idx < 2 * 64 * 64; idx += kAdjThreads) {
        const int c = idx >> 12, i = (idx >> 6) & 63, j = idx & 63;
        const double pv = (i < S && j < S) ? op.P[c][((size_t)r * a.Spad + i) * a.Spad + j] : 0.0;
        const float h = to_tf32((float)pv);
        const float l = to_tf32((float)pv - h);
        unsigned char* m = parea + c * 2 * kPBytes + (j >> 5) * kMatBytes;
        sts(m, sw_off(i, j & 31), h);
        sts(m + kPBytes, sw_off(i, j & 31), l);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tmem_sh;

    if (warp == kAdjEpiWarps) {
        // ---- issuing thread ----
        if (lane == 0) {
            bool ok = true;
            for (int t = 0; ok && t < n_tiles; ++t) {
                if (!mbar_wait_or_abort(&a_ready, t & 1, abort_v)) {
                    atomicOr(&abort_sh, 1);
                    break;
                }
                tc_fence_after();
                for (int c = 0; c < 2; ++c) {   // v_c = x_c P_c^T
                    const unsigned char* ph = parea + c * 2 * kPBytes;
                    const uint32_t d = tm + kColV + c * 64;
                    for (int ks = 0; ks < 8; ++ks) {
                        const int koff = (ks >> 2) * kMatBytes + (ks & 3) * 32;
                        const uint64_t bh = sw128_desc(ph + koff);
                        const uint64_t bl = sw128_desc(ph + kPBytes + koff);
                        const uint32_t ax = tm + kColX + c * 64 + ks * 8;
                        mma_tf32_ta(d, ax, bh, ks > 0);
                        mma_tf32_ta(d, ax, bl, 1);
                        if (SPLITX) mma_tf32_ta(d, tm + kColXL + c * 64 + ks * 8, bh, 1);
                    }
                }
                mma_commit(&v_full);
                // M_c += [U_hi; U_lo]^T (x_hi + x_lo), one slice per warp and child
                for (int w = 0; ok && w < kAdjEpiWarps; ++w) {
                    const unsigned char* sl = slices + w * L::slice;
                    for (int c = 0; c < 2; ++c) {
                        const int k = 2 * t + c;
                        if (!mbar_wait_or_abort(&s_full[w], k & 1, abort_v)) {
                            atomicOr(&abort_sh, 2);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tm + kColM + c * 64;
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = sw128_desc(sl + ks * 32);
                            mma_tf32(d, ad, sw128_desc(sl + kStackBytes + ks * 32), 1);
                            if (SPLITX)
                                mma_tf32(d, ad, sw128_desc(sl + kStackBytes + kMatBytes + ks * 32), 1);
                        }
                        mma_commit(&s_empty[w]);
                    }
                }
            }
            // completes once every product issued above has finished
            mma_commit(&done);
        }
        __syncwarp();
    } else {
        // ---- epilogue warps: thread = pattern = TMEM lane ----
        const uint32_t lane_base = tm + ((uint32_t)(warp * 32) << 16);
        const float wr = (float)a.catw[r];
        unsigned char* sl = slices + warp * L::slice;
        {
            float z[64];
#pragma unroll
            for (int i = 0; i < 64; ++i) z[i] = 0.f;
            tmem_st64(lane_base + kColM, z);
            tmem_st64(lane_base + kColM + 64, z);
        }
        for (int t = 0; t < n_tiles; ++t) {
            const int p = p_begin + t * kTcM + warp * 32 + lane;
            const size_t off = ((size_t)r * a.Ppad + p) * 64;
            // A of the first product: this pattern's x_a, x_b rows (hi, lo)
            for (int c = 0; c < 2; ++c) {
                float x[64];
                if (op.st[c]) {
                    const int s = op.st[c][p];
                    const bool amb = s < 0 || s >= S;
#pragma unroll
                    for (int j = 0; j < 64; ++j) x[j] = (j < S && (amb || s == j)) ? 1.f : 0.f;
                } else {
                    load_row(op.part[c] + off, x);
                }
                if (SPLITX) {
                    float lo[64];
#pragma unroll
                    for (int j = 0; j < 64; ++j) {
                        const float h = to_tf32(x[j]);
                        lo[j] = to_tf32(x[j] - h);
                        x[j] = h;
                    }
                    tmem_st64(lane_base + kColXL + c * 64, lo);
                }
                tmem_st64(lane_base + kColX + c * 64, x);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_ready);
            // q and the pattern's coefficient while the first product runs
            float q[64];
            if (op.q) {
                load_row(op.q + off, q);
            } else {
#pragma unroll
                for (int j = 0; j < 64; ++j) q[j] = j < S ? (float)a.pi[j] : 0.f;
            }
            const float cf = (float)a.coef[(size_t)blockIdx.x * a.Ppad + p] * wr;
            const bool live = cf != 0.f;   // padded and zero-weight patterns add nothing
            const bool got = mbar_wait_or_abort(&v_full, t & 1, abort_v);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) atomicOr(&abort_sh, 4);
                break;
            }
            tc_fence_after();
            bool ok = true;
            for (int c = 0; c < 2; ++c) {
                const int k = 2 * t + c;
                if (k > 0) {   // the products that read this slice last are done
                    const bool fr = mbar_wait_or_abort(&s_empty[warp], (k - 1) & 1, abort_v);
                    if (!__all_sync(0xffffffffu, fr)) {
                        if (lane == 0) atomicOr(&abort_sh, 8);
                        ok = false;
                        break;
                    }
                }
                // U_c = coef w_r q o v_sibling, as TF32 hi (rows 0-63) and lo (64-127)
                float u[64];
                tmem_ld64(lane_base + kColV + (1 - c) * 64, u);
#pragma unroll
                for (int i = 0; i < 64; ++i) {
                    const float val = live ? cf * q[i] * u[i] : 0.f;
                    const float h = to_tf32(val);
                    sts(sl, sw_off(i, lane), h);
                    sts(sl, sw_off(64 + i, lane), to_tf32(val - h));
                }
                // x_c^T (hi; lo with split partials), column = this pattern
                float x[64];
                tmem_ld64(lane_base + kColX + c * 64, x);
#pragma unroll
                for (int j = 0; j < 64; ++j) sts(sl + kStackBytes, sw_off(j, lane), live ? x[j] : 0.f);
                if (SPLITX) {
                    tmem_ld64(lane_base + kColXL + c * 64, x);
#pragma unroll
                    for (int j = 0; j < 64; ++j)
                        sts(sl + kStackBytes + kMatBytes, sw_off(j, lane), live ? x[j] : 0.f);
                }
                fence_proxy_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_full[warp]);
            }
            if (!ok) break;
        }
        // every product has finished (a bounded wait on elapsed time only:
        // TMEM is released below, so products still running must end first)
        const bool fin = __all_sync(0xffffffffu, mbar_wait(&done, 0));
        tc_fence_after();
        const bool good = fin && __all_sync(0xffffffffu, *abort_v == 0);
        // lanes 64-127 hold U_lo^T x: staged in the (now idle) matrix area
        // and added to U_hi^T x of lanes 0-63
        float* stage = reinterpret_cast<float*>(parea);   // [2][64][65]
        if (good && warp >= 2) {
            for (int c = 0; c < 2; ++c) {
                float mv[64];
                tmem_ld64(lane_base + kColM + c * 64, mv);
                float* row = stage + ((size_t)c * 64 + (warp - 2) * 32 + lane) * 65;
#pragma unroll
                for (int j = 0; j < 64; ++j) row[j] = mv[j];
            }
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * kAdjEpiWarps) : "memory");
        if (good && warp < 2) {
            const int i = warp * 32 + lane;
            for (int c = 0; c < 2; ++c) {
                float mv[64];
                tmem_ld64(lane_base + kColM + c * 64, mv);
                const int row = op.row[c];
                if (row < 0) continue;
                const float* srow = stage + ((size_t)c * 64 + i) * 65;
                double* dst = mpart + (size_t)blockIdx.z * a.n_rows +
                              (size_t)(row * a.R + r) * 4096 + (size_t)i * 64;
#pragma unroll 8
                for (int j = 0; j < 64; ++j) dst[j] = (double)mv[j] + (double)srow[j];
            }
        }
        if (!good && warp == 0 && lane == 0) atomicOr(a.timeout, (1 << 11) | (*abort_v & 0xff) | 16);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kAdjEpiWarps) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tm),
                     "r"(kAdjTmemCols)
                     : "memory");
    }
}

}  // namespace

int launch_adj_tc(Instance* I, const AdjOp<float>* d_ops, int n_ops, int n_chunks,
                  const AdjArgs& a, double* d_mpart) {
    const dim3 grid(n_ops, I->R, n_chunks);
    if (n_ops == 0) return TL_OK;
    if (I->split_partials) {
        const size_t smem = AdjTcLayout<true>::smem;
        cudaFuncSetAttribute(k_adj_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_adj_tc<true><<<grid, kAdjThreads, smem, I->stream>>>(d_ops, a, d_mpart);
    } else {
        const size_t smem = AdjTcLayout<false>::smem;
        cudaFuncSetAttribute(k_adj_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_adj_tc<false><<<grid, kAdjThreads, smem, I->stream>>>(d_ops, a, d_mpart);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "adjoint (tensor cores)");
}

}  // namespace tl
