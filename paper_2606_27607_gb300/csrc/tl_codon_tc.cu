// Codon (61 states, padded to 64) post-order pruning on the 5th-generation
// tensor cores: tcgen05.mma kind::tf32 with TMEM accumulators and TMA-staged,
// 128-byte-swizzled operands.
//
// For a child c and rate category r the update is a dense contraction over
// the child's states, v_c[p, i] = sum_j x_c[p, j] P_c,r[i, j] (Sec.
// "Introduction": pruning; Sec. "Tensor cores": likelihoods as GEMMs for
// large state spaces). With the child partials as A (M = 128 patterns x
// K = 64 states, K-major) and P as B (N = 64 output states x K = 64, K-major,
// i.e. P row-major) one M128 N64 K64 product per (child, category) lands in
// its own 64-column block of tensor memory (2 children x 4 categories = 512
// columns). The epilogue (all 128 threads, one TMEM lane = one pattern)
// multiplies the two children, takes the per-pattern maximum over categories
// and states, rescales by a power of two, rounds to TF32 and stores. A tip
// child with a state code is a column of P: a row of the TF32-rounded P^T
// copy, read directly (no MMA). Partials are stored TF32-rounded, so the
// tensor core reads exactly the stored values.
//
// Work items are (op, 128-pattern tile) pairs of one tree level; thread 0
// runs a 4-stage TMA -> MMA pipeline on mbarriers; every wait is bounded and
// sets an error flag instead of hanging.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "tl_internal.cuh"

namespace tl {
namespace {

constexpr int kTcM = 128;                   // patterns per tile (TMEM lanes)
constexpr int kTcN = 64;                    // padded states
constexpr int kStages = 4;
constexpr int kAChunk = kTcM * 32 * 4;      // 32 K-values of 128 rows: 16 KB
constexpr int kBChunk = kTcN * 32 * 4;      // 8 KB
constexpr int kStageBytes = 2 * kAChunk + 2 * kBChunk;  // 48 KB
constexpr int kTmemCols = 512;
constexpr unsigned kSpinLimit = 1u << 22;   // bounded mbarrier waits

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Wait for the phase with the given parity; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;           // start address
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}
// Instruction descriptor: D f32, A and B tf32, both K-major, N = 64, M = 128.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((kTcN >> 3) << 17) |
                                ((kTcM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdescTf32), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ int frexp_exp_f(float m) {
    int E = (__float_as_int(m) >> 23) & 0xff;
    if (E == 0) {
        if (m == 0.f) return 0;
        E = ((__float_as_int(m * 18446744073709551616.f) >> 23) & 0xff) - 64;
    }
    return E - 126;
}
__device__ __forceinline__ float pow2f(int k) {  // 2^k, k in [-126, 127]
    return __int_as_float((k + 127) << 23);
}

// ---- device op descriptor ----------------------------------------------------
struct __align__(16) TcOp {
    int child[2];
    int kind[2];      // kInternal (pool), kTipPartials (tip pool), kTipStates (lookup)
    int mat[2];
    int dest;
    int pad;
};

struct TcArgs {
    float* pool;              // [n_buffers][R][Ppad][64]
    int* epool;               // [n_buffers][Ppad]
    const int8_t* tips;       // [n_tips][Ppad]
    const float* matw;        // [slot][2][R][64][64]: P, then P^T (TF32-rounded)
    const float* rowsum;      // [slot][R][64]
    int R, Ppad, S, n_tiles, rescale;
    size_t bstride;           // floats per buffer
    int* err;
};

// One level of post-order ops; items = n_ops * n_tiles.
__global__ void __launch_bounds__(128, 1)
k_post_tc(const __grid_constant__ CUtensorMap tm_part, const __grid_constant__ CUtensorMap tm_tip,
          const __grid_constant__ CUtensorMap tm_mat, const TcOp* __restrict__ ops, int n_ops,
          TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    // 128-byte swizzle atoms must start on 1024-byte shared-memory addresses
    unsigned char* stages = smem_tc + ((1024u - (smem_u32(smem_tc) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    __shared__ unsigned produced_sh, consumed_sh;
    const int tid = threadIdx.x, warp = tid >> 5;

    if (warp == 0) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                smem_u32(&tmem_base_sh)),
            "r"(kTmemCols)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_sh = 0;
        produced_sh = consumed_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int R = a.R;
    unsigned pairs_done = 0;   // (child, category) products issued by this CTA
    unsigned items_done = 0;   // items with at least one product

    const int n_items = n_ops * a.n_tiles;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int k = item / a.n_tiles, tile = item % a.n_tiles;
        const TcOp op = ops[k];
        const int p0 = tile * kTcM;
        // "internal" = contracted on the tensor cores (pool or tip-partials A)
        const bool internal[2] = {op.kind[0] != kTipStates, op.kind[1] != kTipStates};
        const int n_pairs = (internal[0] + internal[1]) * R;
        if (tid == 0 && n_pairs > 0) {
            // software pipeline: produce pair i, consume pair i - (kStages - 1)
            bool ok = true;
            int produced = 0, consumed = 0;
            for (int i = 0; ok && i < n_pairs + kStages - 1; ++i) {
                if (i < n_pairs) {
                    const unsigned g = pairs_done + i;
                    const int s = g % kStages;
                    const unsigned round = g / kStages;
                    ok = mbar_wait(&empty[s], (round & 1) ^ 1);
                    if (!ok) break;
                    const int c = internal[0] ? (i < R ? 0 : 1) : 1;
                    const int r = i % R;
                    unsigned char* st = stages + s * kStageBytes;
                    mbar_expect_tx(&full[s], kStageBytes);
                    const int arow = (op.child[c] * R + r) * a.Ppad + p0;
                    const int brow = (op.mat[c] * 2 * R + r) * kTcN;
                    const CUtensorMap* am = op.kind[c] == kTipPartials ? &tm_tip : &tm_part;
                    tma_load_2d(st, am, 0, arow, &full[s]);
                    tma_load_2d(st + kAChunk, am, 32, arow, &full[s]);
                    tma_load_2d(st + 2 * kAChunk, &tm_mat, 0, brow, &full[s]);
                    tma_load_2d(st + 2 * kAChunk + kBChunk, &tm_mat, 32, brow, &full[s]);
                    ++produced;
                }
                const int j = i - (kStages - 1);
                if (j >= 0) {
                    const unsigned g = pairs_done + j;
                    const int s = g % kStages;
                    ok = mbar_wait(&full[s], (g / kStages) & 1);
                    if (!ok) break;
                    tc_fence_after();
                    const int c = internal[0] ? (j < R ? 0 : 1) : 1;
                    const int r = j % R;
                    const uint32_t d = tmem + (uint32_t)(r * 2 * kTcN + c * kTcN);
                    unsigned char* st = stages + s * kStageBytes;
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks) {
                        const int chunk = ks >> 2, kin = (ks & 3) * 32;
                        const uint64_t ad = sw128_desc(st + chunk * kAChunk + kin);
                        const uint64_t bd = sw128_desc(st + 2 * kAChunk + chunk * kBChunk + kin);
                        mma_tf32(d, ad, bd, ks > 0 ? 1u : 0u);
                    }
                    mma_commit(&empty[s]);
                    ++consumed;
                }
            }
            mma_commit(&done);
            if (!ok) abort_sh = 1;
            produced_sh = pairs_done + produced;
            consumed_sh = pairs_done + consumed;
        }
        __syncthreads();
        bool fail = abort_sh != 0;
        if (!fail && n_pairs > 0) fail = !mbar_wait(&done, items_done & 1);
        if (__syncthreads_or(fail)) {
            abort_sh = 1;
            break;
        }
        if (n_pairs > 0) {
            tc_fence_after();
            ++items_done;
        }
        pairs_done += n_pairs;

        // ---- epilogue: lane tid <-> pattern p0 + tid -----------------------
        const int p = p0 + tid;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const float* col[2] = {nullptr, nullptr};
        bool amb[2] = {false, false};
        int cum = 0;
        for (int c = 0; c < 2; ++c) {
            if (!internal[c]) {
                const int s = a.tips[(size_t)op.child[c] * a.Ppad + p];
                amb[c] = !(s >= 0 && s < a.S);
                col[c] = !amb[c]
                             ? a.matw + (((size_t)op.mat[c] * 2 + 1) * R) * kTcN * kTcN + (size_t)s * kTcN
                             : a.rowsum + (size_t)op.mat[c] * R * kTcN;
            } else if (op.kind[c] == kInternal) {
                cum += a.epool[(size_t)op.child[c] * a.Ppad + p];
            }
        }
        // child value chunk (16 states, category r)
        auto chunk = [&](int c, int r, int q, float* v) {
            if (internal[c]) {
                tmem_ld16(lane_base + (uint32_t)(r * 2 * kTcN + c * kTcN + q * 16), v);
            } else {
                const size_t rstride = amb[c] ? kTcN : kTcN * kTcN;
                const float4* src = reinterpret_cast<const float4*>(col[c] + r * rstride + q * 16);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 f = __ldg(src + u);
                    v[4 * u] = f.x;
                    v[4 * u + 1] = f.y;
                    v[4 * u + 2] = f.z;
                    v[4 * u + 3] = f.w;
                }
            }
        };
        float m = 0.f;
        for (int r = 0; r < R; ++r)
            for (int q = 0; q < 4; ++q) {
                float x[16], y[16];
                chunk(0, r, q, x);
                chunk(1, r, q, y);
#pragma unroll
                for (int i = 0; i < 16; ++i) m = fmaxf(m, x[i] * y[i]);
            }
        int e = a.rescale ? frexp_exp_f(m) : 0;
        float f1 = 1.f, f2 = 1.f;
        if (e != 0) {
            const int kk = -e;
            if (kk >= -126 && kk <= 126) f1 = pow2f(kk);
            else {
                f1 = pow2f(kk / 2);
                f2 = pow2f(kk - kk / 2);
            }
            cum += e;
        }
        float* dst = a.pool + (size_t)op.dest * a.bstride + (size_t)p * kTcN;
        for (int r = 0; r < R; ++r)
            for (int q = 0; q < 4; ++q) {
                float x[16], y[16];
                chunk(0, r, q, x);
                chunk(1, r, q, y);
                float4* o = reinterpret_cast<float4*>(dst + (size_t)r * a.Ppad * kTcN + q * 16);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    float4 w;
                    w.x = to_tf32(x[4 * u] * y[4 * u] * f1 * f2);
                    w.y = to_tf32(x[4 * u + 1] * y[4 * u + 1] * f1 * f2);
                    w.z = to_tf32(x[4 * u + 2] * y[4 * u + 2] * f1 * f2);
                    w.w = to_tf32(x[4 * u + 3] * y[4 * u + 3] * f1 * f2);
                    o[u] = w;
                }
            }
        a.epool[(size_t)op.dest * a.Ppad + p] = cum;
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (abort_sh && tid == 0) {
        atomicOr(a.err, 4);
        // bounded drain of copies and products still in flight
        for (unsigned g = consumed_sh; g < produced_sh; ++g)
            mbar_wait(&full[g % kStages], (g / kStages) & 1);
        mbar_wait(&done, items_done & 1);
    }
    // no MMA may still write TMEM when it is released
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

// Root log-likelihood of a TF32 instance: thread per pattern, block partial
// sums (fixed order).
__global__ void k_root_tc(const float* __restrict__ x, const int* __restrict__ ep,
                          const double* __restrict__ pi, TcArgs a, const double* __restrict__ patw,
                          int P, double* __restrict__ site, double* __restrict__ part,
                          const double* __restrict__ catw) {
    __shared__ double wsum[32];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (p < a.Ppad) {
        double L = 0.0;
        for (int r = 0; r < a.R; ++r) {
            const float* v = x + ((size_t)r * a.Ppad + p) * kTcN;
            double s = 0.0;
            for (int q = 0; q < a.S; ++q) s += pi[q] * (double)v[q];
            L += catw[r] * s;
        }
        const double l = log(L) + 0.69314718055994530942 * (double)(ep ? ep[p] : 0);
        if (p < P) {
            if (!(L > 0.0) || !isfinite(l)) atomicOr(a.err, 1);
            if (site) site[p] = l;
            contrib = patw[p] * l;
        }
    }
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = contrib;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        part[blockIdx.x] = t;
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map over rows of 64 floats, box 32 x box_rows, 128-byte swizzle.
int make_map(Instance* I, CUtensorMap* m, void* base, size_t rows, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return fail(I, TL_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[2] = {(cuuint64_t)kTcN, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kTcN * sizeof(float)};
    cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(I, TL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TL_OK;
}

TcArgs tc_args(Instance* I) {
    TcArgs a;
    a.pool = reinterpret_cast<float*>(I->pool);
    a.epool = I->scale_pool;
    a.tips = I->tip_pool;
    a.matw = reinterpret_cast<const float*>(I->d_matw);
    a.rowsum = I->d_rowsum;
    a.R = I->R;
    a.Ppad = I->Ppad;
    a.S = I->S;
    a.n_tiles = I->Ppad / kTcM;
    a.rescale = I->rescale;
    a.bstride = (size_t)I->R * I->Ppad * kTcN;
    a.err = I->d_err + 2;
    return a;
}

}  // namespace

int tc_tile() { return kTcM; }

int tc_setup(Instance* I) {
    static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
    I->tmaps.resize(3 * sizeof(CUtensorMap));
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(I->tmaps.data());
    int rc;
    const size_t rows = (size_t)I->n_buffers * I->R * I->Ppad;
    if ((rc = make_map(I, &m[0], I->pool, rows, kTcM))) return rc;
    if ((rc = make_map(I, &m[2], I->d_matw, (size_t)I->n_mats * 2 * I->R * kTcN, kTcN))) return rc;
    m[1] = m[0];  // tip-partials map until a tip pool exists
    return TL_OK;
}

int tc_set_tip_pool(Instance* I) {
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(I->tmaps.data());
    return make_map(I, &m[1], I->tc_tip_pool, (size_t)I->n_tips * I->R * I->Ppad, kTcM);
}

int launch_post_tc(Instance* I, const tl_op* ops, int n, void* d_ops_area, size_t cap) {
    // tree levels: an op runs after the ops that produce its children
    std::vector<int> producer(I->n_bufs, -1), level(n, 0);
    for (int k = 0; k < n; ++k) {
        const int ch[2] = {ops[k].child1, ops[k].child2};
        for (int c = 0; c < 2; ++c)
            if (ch[c] >= I->n_tips && producer[ch[c]] >= 0)
                level[k] = std::max(level[k], level[producer[ch[c]]] + 1);
        producer[ops[k].dest] = k;
    }
    const int n_levels = n ? *std::max_element(level.begin(), level.end()) + 1 : 0;
    std::vector<TcOp> dev;
    std::vector<int> first(n_levels + 1, 0);
    dev.reserve(n);
    for (int L = 0; L < n_levels; ++L) {
        first[L] = (int)dev.size();
        for (int k = 0; k < n; ++k) {
            if (level[k] != L) continue;
            TcOp t;
            std::memset(&t, 0, sizeof t);
            const int ch[2] = {ops[k].child1, ops[k].child2};
            const int mt[2] = {ops[k].mat1, ops[k].mat2};
            for (int c = 0; c < 2; ++c) {
                t.mat[c] = mt[c];
                if (ch[c] < I->n_tips) {
                    t.kind[c] = I->tip_set[ch[c]] == 1 ? kTipStates : kTipPartials;
                    t.child[c] = ch[c];
                } else {
                    t.kind[c] = kInternal;
                    t.child[c] = ch[c] - I->n_tips;
                }
            }
            t.dest = ops[k].dest - I->n_tips;
            dev.push_back(t);
        }
    }
    first[n_levels] = (int)dev.size();
    if (dev.size() * sizeof(TcOp) > cap) return fail(I, TL_ERR_ARG, "op area too small");
    int rc = upload_bytes(I, d_ops_area, dev.data(), dev.size() * sizeof(TcOp));
    if (rc) return rc;
    const size_t smem = (size_t)kStages * kStageBytes + 1024;
    cudaFuncSetAttribute(k_post_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int sms = 0, dev_id = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(I->tmaps.data());
    TcArgs a = tc_args(I);
    const TcOp* d = reinterpret_cast<const TcOp*>(d_ops_area);
    for (int L = 0; L < n_levels; ++L) {
        const int nl = first[L + 1] - first[L];
        const int items = nl * a.n_tiles;
        const int grid = std::max(1, std::min(items, sms));
        k_post_tc<<<grid, 128, smem, I->stream>>>(m[0], m[1], m[2], d + first[L], nl, a);
        I->launches += 1;
    }
    return cuda_check(I, cudaGetLastError(), "tensor-core post-order kernel");
}

int launch_root_tc(Instance* I, int root_pool, int model, double* d_site, double* d_part,
                   int n_parts) {
    TcArgs a = tc_args(I);
    const float* x = a.pool + (size_t)root_pool * a.bstride;
    const int* ep = a.epool + (size_t)root_pool * a.Ppad;
    double* catw = I->d_tmp;  // staged by the caller
    k_root_tc<<<n_parts, 128, 0, I->stream>>>(x, ep, I->models[model].pi, a, I->d_patw, I->P,
                                              d_site, d_part, catw);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "tensor-core root kernel");
}

}  // namespace tl
