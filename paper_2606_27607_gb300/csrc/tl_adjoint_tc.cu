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
// patterns, eight epilogue warps and one issuing warp. Two epilogue warps
// share a TMEM lane quarter (thread = pattern = lane) and split the states
// between them (columns 0-31 and 32-63); each thread loads the next tile's
// rows while the current tile's products run.
//
// First product: A = x_c from tensor memory (each thread stores its half of
// its pattern's row; with split partials also x_lo), B = P_c hi and lo
// (K-major, 128-byte swizzle, resident for the whole chunk): v_c = x P_hi^T
// + x P_lo^T (+ x_lo P_hi^T), M = 128 patterns, N = 64, K = 64.
//
// Second product: the contraction runs over patterns, and a tf32 operand
// must be K-major (its 32-bit elements contiguous along K), so each lane
// quarter writes its 32 patterns transposed: the A operand stacks U_hi^T
// (rows 0-63) over U_lo^T (rows 64-127), one M = 128 operand, and B is x_c^T
// (x_hi^T, with split partials also x_lo^T). The accumulator then holds
// U_hi^T x and U_lo^T x in lanes 0-63 and 64-127, added when the chunk
// ends; one M = 128 instruction per K step carries both halves of the
// split. Each lane quarter owns its transposed slice (32 patterns = one
// 128-byte K chunk), written by its two warps (rows of their states), so
// the four quarters write in parallel and the issuing thread consumes the
// slices in a fixed order.
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

constexpr int kAdjEpiWarps = 8;                 // two per TMEM lane quarter
constexpr int kAdjIssueWarp = kAdjEpiWarps;     // allocates TMEM, issues the products
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
    static constexpr int q_stage = kTcM * 64 * 4;     // the next tile's q, 32 KB
    static constexpr size_t bytes =
        (size_t)p_area + 4 * (size_t)slice + q_stage;   // a slice per lane quarter
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
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// 32 floats of global memory (one 128-byte line).
__device__ __forceinline__ void load_half(const float* src, float* v) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4 f[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) f[u] = s4[u];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
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
    float* qstage = reinterpret_cast<float*>(slices + 4 * L::slice);   // [128][64]
    __shared__ __align__(8) uint64_t xa_ready, xb_ready, v_full[2], s_full[4], s_empty[4], done;
    __shared__ uint32_t tmem_sh;
    __shared__ int abort_sh;  // bit 0 x ready, 1 s_full, 2 v_full, 3 s_empty
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_v = &abort_sh;
    const AdjOp<float>& op = ops[blockIdx.x];
    const int r = blockIdx.y, S = a.S;
    const int p_begin = blockIdx.z * a.chunk;
    const int p_end = min(a.Ppad, p_begin + a.chunk);
    const int n_tiles = p_end > p_begin ? (p_end - p_begin) / kTcM : 0;

    if (tid == 0) {
        abort_sh = 0;
        mbar_init(&xa_ready, kAdjEpiWarps);
        mbar_init(&xb_ready, kAdjEpiWarps);
        mbar_init(&v_full[0], 1);
        mbar_init(&v_full[1], 1);
        for (int w = 0; w < 4; ++w) {
            mbar_init(&s_full[w], 2);   // the two warps of a lane quarter
            mbar_init(&s_empty[w], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == kAdjIssueWarp) {
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

    // TMEM column region (0 or 1, 64 columns each) of x_c for tile t: x_a(t) in
    // region t & 1, x_b(t) in the other, so that x_b(t + 1) can go where
    // x_a(t) was as soon as child a's slice of tile t is written, and x_a(t + 1)
    // where x_b(t) was after child b's slice
    auto xreg = [](int t, int c) -> uint32_t { return (uint32_t)(((t + c) & 1) * 64); };

    if (warp == kAdjIssueWarp) {
        // ---- issuing thread ----
        if (lane == 0) {
            // v_c(t) = x_c(t) P_c^T into its TMEM columns
            auto first_product = [&](int t, int c) {
                const unsigned char* ph = parea + c * 2 * kPBytes;
                const uint32_t d = tm + kColV + c * 64;
                const uint32_t xa = tm + kColX + xreg(t, c), xl = tm + kColXL + xreg(t, c);
                for (int ks = 0; ks < 8; ++ks) {
                    const int koff = (ks >> 2) * kMatBytes + (ks & 3) * 32;
                    const uint64_t bh = sw128_desc(ph + koff);
                    const uint64_t bl = sw128_desc(ph + kPBytes + koff);
                    mma_tf32_ta(d, xa + ks * 8, bh, ks > 0);
                    mma_tf32_ta(d, xa + ks * 8, bl, 1);
                    if (SPLITX) mma_tf32_ta(d, xl + ks * 8, bh, 1);
                }
                mma_commit(&v_full[c]);
            };
            // M_c += [U_hi; U_lo]^T (x_hi + x_lo) for the four quarters' slices
            auto second_product = [&](int t, int c) -> bool {
                for (int w = 0; w < 4; ++w) {
                    const unsigned char* sl = slices + w * L::slice;
                    if (!mbar_wait_or_abort(&s_full[w], (2 * t + c) & 1, abort_v)) {
                        atomicOr(&abort_sh, 2);
                        return false;
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
                return true;
            };
            auto x_ready = [&](int t, int c) -> bool {
                if (!mbar_wait_or_abort(c == 0 ? &xa_ready : &xb_ready, t & 1, abort_v)) {
                    atomicOr(&abort_sh, 1);
                    return false;
                }
                tc_fence_after();
                return true;
            };
            // the order in which the epilogue produces its inputs: x_b(0),
            // x_a(0), then per tile slices a(t), x_b(t+1), slices b(t), x_a(t+1)
            bool ok = n_tiles == 0 || (x_ready(0, 1) && (first_product(0, 1), x_ready(0, 0)));
            if (ok && n_tiles > 0) first_product(0, 0);
            for (int t = 0; ok && t < n_tiles; ++t) {
                const bool more = t + 1 < n_tiles;
                ok = second_product(t, 0);
                if (ok && more && (ok = x_ready(t + 1, 1))) first_product(t + 1, 1);
                if (ok) ok = second_product(t, 1);
                if (ok && more && (ok = x_ready(t + 1, 0))) first_product(t + 1, 0);
            }
            // completes once every product issued above has finished
            mma_commit(&done);
        }
        __syncwarp();
    } else {
        // ---- epilogue: lane quarter qd (thread = pattern = TMEM lane), states
        // [col0, col0 + 32) ----
        const int qd = warp & 3, col0 = (warp >> 2) * 32;
        const uint32_t lane_base = tm + ((uint32_t)(qd * 32) << 16);
        const float wr = (float)a.catw[r];
        unsigned char* sl = slices + qd * L::slice;
        {
            float z[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) z[i] = 0.f;
            tmem_st32(lane_base + kColM + col0, z);
            tmem_st32(lane_base + kColM + 64 + col0, z);
        }
        // this thread's half row of x_c for tile t (one-hot for a tip state)
        auto load_x = [&](int t, int c, float* x) {
            const int p = p_begin + t * kTcM + qd * 32 + lane;
            if (op.st[c]) {
                const int s = op.st[c][p];
                const bool amb = s < 0 || s >= S;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    x[j] = (col0 + j < S && (amb || s == col0 + j)) ? 1.f : 0.f;
            } else {
                load_half(op.part[c] + ((size_t)r * a.Ppad + p) * 64 + col0, x);
            }
        };
        // A of the first product: x_c(t) (hi; lo with split partials) into
        // its TMEM region, then the arrival the issuing thread waits for
        auto put_x = [&](int t, int c, float* x) {
            if (SPLITX) {   // hi = x truncated to TF32, lo = x - hi (exact)
                float lo[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float h = tf32_trunc(x[j]);
                    lo[j] = x[j] - h;
                    x[j] = h;
                }
                tmem_st32(lane_base + kColXL + xreg(t, c) + col0, lo);
            }
            tmem_st32(lane_base + kColX + xreg(t, c) + col0, x);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(c == 0 ? &xa_ready : &xb_ready);
        };
        // q of tile t: this thread's half row copied asynchronously into the
        // stage (16-byte unit u at u ^ (lane & 7), so that the row-per-thread
        // reads below are conflict-free), and the pattern's coefficient
        float* qrow = qstage + (size_t)(qd * 32 + lane) * 64 + col0;
        float cf = 0.f;
        auto fetch_q = [&](int t) {
            const int p = p_begin + t * kTcM + qd * 32 + lane;
            if (op.q) {
                const float* src = op.q + ((size_t)r * a.Ppad + p) * 64 + col0;
#pragma unroll
                for (int u = 0; u < 8; ++u) cp_async16(qrow + 4 * (u ^ (lane & 7)), src + 4 * u);
                cp_async_commit();
            }
            cf = (float)a.coef[(size_t)blockIdx.x * a.Ppad + p] * wr;
        };
        // coef w_r q (padded and zero-weight patterns have coef 0 and finite
        // q, v and x, so they add nothing)
        auto read_q = [&](float* q) {
            if (op.q) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 f = *reinterpret_cast<const float4*>(qrow + 4 * (u ^ (lane & 7)));
                    q[4 * u] = cf * f.x;
                    q[4 * u + 1] = cf * f.y;
                    q[4 * u + 2] = cf * f.z;
                    q[4 * u + 3] = cf * f.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) q[j] = col0 + j < S ? cf * (float)a.pi[col0 + j] : 0.f;
            }
        };
        // Element (col0 + i, lane) of a 128-byte-swizzled slice part sits at
        // row base(i & 7) + part + i * 128: the stores below run by row phase
        // k = i & 7, one base per phase, the rest immediate offsets.
        unsigned char* const colbase = sl + col0 * 128 + (lane & 3) * 4;
        auto store32 = [&](int part, const float* v) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                // the 16-byte unit of this lane's column in rows of phase k
                unsigned char* b = colbase + ((((lane >> 2) ^ k) & 7) << 4) + part;
#pragma unroll
                for (int i = k; i < 32; i += 8) *reinterpret_cast<float*>(b + i * 128) = v[i];
            }
        };
        // wait for a barrier phase in every lane, or record where it gave up
        auto wait_all = [&](uint64_t* bar, unsigned parity, int bit) -> bool {
            const bool got = mbar_wait_or_abort(bar, parity, abort_v);
            if (__all_sync(0xffffffffu, got)) return true;
            if (lane == 0) atomicOr(&abort_sh, bit);
            return false;
        };
        // child c's slice of tile t: U_c = coef w_r q o v_sibling as TF32 hi
        // (rows i) and lo (rows 64 + i), and x_c^T (hi; lo), column = pattern
        auto slice = [&](int t, int c) -> bool {
            const int k = 2 * t + c;
            if (k > 0 && !wait_all(&s_empty[qd], (k - 1) & 1, 8)) return false;
            float q[32], u[32];
            read_q(q);
            // the stage is free once child b has read q(t): q(t + 1) copies in
            // while this slice and the next x are written
            if (c == 1 && t + 1 < n_tiles) fetch_q(t + 1);
            tmem_ld32(lane_base + kColV + (1 - c) * 64 + col0, u);
            // hi = U truncated to TF32 (rows i), lo = U - hi (rows 64 + i, exact;
            // the tensor core reads its leading 11 bits)
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float val = q[i] * u[i];
                q[i] = tf32_trunc(val);
                u[i] = val - q[i];
            }
            store32(0, q);
            store32(64 * 128, u);
            tmem_ld32(lane_base + kColX + xreg(t, c) + col0, u);
            store32(kStackBytes, u);
            if (SPLITX) {
                tmem_ld32(lane_base + kColXL + xreg(t, c) + col0, u);
                store32(kStackBytes + kMatBytes, u);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_full[qd]);
            return true;
        };
        float xn[32];
        if (n_tiles > 0) {
            fetch_q(0);
            load_x(0, 1, xn);
            put_x(0, 1, xn);
            load_x(0, 0, xn);
            put_x(0, 0, xn);
        }
        for (int t = 0; t < n_tiles; ++t) {
            const bool more = t + 1 < n_tiles;
            // the next tile's x_b, in flight during child a's slice
            if (more) load_x(t + 1, 1, xn);
            cp_async_wait_all();   // this thread's q(t)
            // child a: needs v_b(t); its slice frees x_a(t)'s region
            if (!wait_all(&v_full[1], t & 1, 4)) break;
            tc_fence_after();
            if (!slice(t, 0)) break;
            // v_a(t) is done reading x_a(t)'s region before x_b(t + 1) goes there
            if (!wait_all(&v_full[0], t & 1, 4)) break;
            tc_fence_after();
            if (more) {
                put_x(t + 1, 1, xn);
                load_x(t + 1, 0, xn);   // in flight during child b's slice
            }
            if (!slice(t, 1)) break;
            if (more) put_x(t + 1, 0, xn);
        }
        cp_async_wait_all();
        // every product has finished (a bounded wait on elapsed time only:
        // TMEM is released below, so products still running must end first)
        const bool fin = __all_sync(0xffffffffu, mbar_wait(&done, 0));
        tc_fence_after();
        const bool good = fin && __all_sync(0xffffffffu, *abort_v == 0);
        // lanes 64-127 hold U_lo^T x: staged in the (now idle) matrix area
        // and added to U_hi^T x of lanes 0-63
        float* stage = reinterpret_cast<float*>(parea);   // [2][64][65]
        if (good && qd >= 2) {
            for (int c = 0; c < 2; ++c) {
                float mv[32];
                tmem_ld32(lane_base + kColM + c * 64 + col0, mv);
                float* row = stage + ((size_t)c * 64 + (qd - 2) * 32 + lane) * 65 + col0;
#pragma unroll
                for (int j = 0; j < 32; ++j) row[j] = mv[j];
            }
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(32 * kAdjEpiWarps) : "memory");
        if (good && qd < 2) {
            const int i = qd * 32 + lane;
            for (int c = 0; c < 2; ++c) {
                float mv[32];
                tmem_ld32(lane_base + kColM + c * 64 + col0, mv);
                const int row = op.row[c];
                if (row < 0) continue;
                const float* srow = stage + ((size_t)c * 64 + i) * 65 + col0;
                double* dst = mpart + (size_t)blockIdx.z * a.n_rows +
                              (size_t)(row * a.R + r) * 4096 + (size_t)i * 64 + col0;
#pragma unroll 8
                for (int j = 0; j < 32; ++j) dst[j] = (double)mv[j] + (double)srow[j];
            }
        }
        if (!good && warp == 0 && lane == 0) atomicOr(a.timeout, (1 << 11) | (*abort_v & 0xff) | 16);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kAdjIssueWarp) {
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
