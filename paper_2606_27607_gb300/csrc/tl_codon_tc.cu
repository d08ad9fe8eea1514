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
#include "tl_tcgen05.cuh"

namespace tl {
namespace {
using namespace tc5;

constexpr int kStages = 4;                  // most pipeline stages (barrier arrays)
constexpr int kAChunk = kTcM * 32 * 4;      // 32 K-values of 128 rows: 16 KB
constexpr int kBChunk = kTcN * 32 * 4;      // 8 KB
// Stage: A (2 x 16 KB) and B (2 x 8 KB) = 48 KB, four stages; with split
// matrices a stage also holds B_lo (64 KB), so three fit; with split
// partials also A_lo (96 KB), two stages.
// Per-warp staging for coalesced stores of the epilogue's rows: 32 half rows.
constexpr int kOutWarpBytes = 32 * 128;
// The level kernels run eight warps: two per TMEM lane quarter (thread =
// pattern = lane), each taking half of the rate categories; per-pattern
// partial results (maxima, sums over categories) meet in shared memory.
constexpr int kTcThreads = 256;

template <bool SPLIT, bool SPLITA>
struct TcPipe {
    static constexpr int stages = SPLITA ? 2 : (SPLIT ? 3 : 4);
    static constexpr int a_bytes = (SPLITA ? 4 : 2) * kAChunk;   // A (and A_lo)
    static constexpr int bytes = a_bytes + (SPLIT ? 4 : 2) * kBChunk;
    // bytes the copies of one stage bring in (A_lo is computed on chip)
    static constexpr int tx_bytes = 2 * kAChunk + (SPLIT ? 4 : 2) * kBChunk;
};
constexpr int kTmemCols = 512;

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
// Post-order partials are stored with their per-pattern maximum (over
// categories and states) in [2^(K-1), 2^K), K = kPostExp. The product of two
// stored children, and the pre-order ratio denominator q . (v_a o v_b)
// formed from them, then sit 2^(2K) above the values a maximum near 1 would
// give: underflow below FP32's smallest normal number needs a normalised
// product below 2^-(126+2K). The largest value any kernel forms from stored
// partials stays below 2^(2K+30) (products of two children, sums over 64
// states and 8 categories, derivative matrices with entries below 2^20).
// Power-of-two scaling commutes with rounding, so every result whose
// intermediates stayed normal is unchanged.
constexpr int kPostExp = 48;
// Factors f1 f2 = 2^(K-e) that bring a maximum m = f 2^e, f in [0.5, 1), to
// [2^(K-1), 2^K) (split in two when out of pow2f's range); returns the
// exponent the stored values omit, e - K (0 for an all-zero pattern).
__device__ __forceinline__ int post_scale(float m, float* f1, float* f2) {
    *f1 = 1.f;
    *f2 = 1.f;
    if (m == 0.f) return 0;
    const int kk = kPostExp - frexp_exp_f(m);
    if (kk >= -126 && kk <= 126) {
        *f1 = pow2f(kk);
    } else {
        *f1 = pow2f(kk / 2);
        *f2 = pow2f(kk - kk / 2);
    }
    return -kk;
}

// ---- device op descriptor ----------------------------------------------------
// Two operands per work item. Operand c is either contracted on the tensor
// cores (A from the partials pool or the tip-partials pool, B from the
// matrix map at rows brow[c] + 64 r) or, for a tip with a state code, looked
// up in a P^T block of the matrix array (look[c], floats, category 0).
struct __align__(16) TcOp {
    int child[2];
    int kind[2];      // kInternal, kTipPartials: MMA; kTipStates: lookup; -1: no operand
    int brow[2];
    int look[2];
    int dest;         // post: output buffer; pre2: q buffer (holds u on entry)
    int qin;          // pre1: parent q buffer, -1 for the root (q = pi)
    int uout[2];      // pre1: buffer receiving u of each internal child (-1: none)
    int edge[2];      // gradient row (-1: none)
    int dlook[2];     // pre1: dP^T block of a tip child (numerator lookup)
};

struct TcArgs {
    float* pool;              // [n_buffers][R][Ppad][64]
    int* epool;               // [n_buffers][Ppad]
    const int8_t* tips;       // [n_tips][Ppad]
    const float* matw;        // [slot][2][R][64][64]: P, then P^T (TF32-rounded); then Q copies
    const float* rowsum;      // [slot][R][64]
    const double* patw;       // [Ppad]
    const double* pi;         // [64] root frequencies (pre1)
    double* gpart;            // [edge rows][n_tiles] gradient partials
    int R, Ppad, S, n_tiles, rescale;
    int dgen;                 // pre2: operand 1 is dP x for any derivative dP (not Q x)
    size_t bstride;           // floats per buffer
    int* err;
    float catw[kMaxCat], rates[kMaxCat];
};

static_assert(sizeof(TcOp) == kTcOpBytes, "descriptor size");

enum TcMode { kPost = 0, kPre1 = 1, kPre2 = 2 };

// Fixed-order sum over the 128 threads; thread 0 gets the total.
// Sum of v over the block's eight warps (fixed order); the result in thread 0.
__device__ __forceinline__ float block_sum256(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        t = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
    __syncthreads();
    return t;
}

// SPLIT: B = B_hi + B_lo, the lo rows 2 R 64 rows after the hi rows of the
// same block (lookups: 2 R 64 64 floats after), and each k-step issues the
// hi and the lo product into the same accumulator.
// SPLITA (with SPLIT): the partials are stored in full FP32, and every A tile
// is split in shared memory, once its copy has landed, into A_hi = the TF32
// truncation (in place) and A_lo = the TF32 truncation of A - A_hi (all 128
// threads, one 16-byte chunk at a time: the split is elementwise, so the
// 128-byte swizzle of the tile does not matter); each k-step issues
// A_hi B_hi + A_hi B_lo + A_lo B_hi, which keeps about 21 bits of both
// operands (the A_lo B_lo term is below FP32 rounding of the sum).
template <int MODE, bool SPLIT, bool SPLITA>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc(const __grid_constant__ CUtensorMap tm_part, const __grid_constant__ CUtensorMap tm_tip,
     const __grid_constant__ CUtensorMap tm_mat, const TcOp* __restrict__ ops, int n_ops,
     TcArgs a) {
    static_assert(!SPLITA || SPLIT, "split partials need split matrices");
    constexpr int kSt = TcPipe<SPLIT, SPLITA>::stages;
    constexpr int kStB = TcPipe<SPLIT, SPLITA>::bytes;
    constexpr int kBOff = TcPipe<SPLIT, SPLITA>::a_bytes;   // B_hi within a stage
    const size_t kLoFloats = (size_t)2 * a.R * kTcN * kTcN;  // hi block -> lo block
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    // 128-byte swizzle atoms must start on 1024-byte shared-memory addresses
    unsigned char* stages = smem_tc + ((1024u - (smem_u32(smem_tc) & 1023u)) & 1023u);
    unsigned char* wout = stages + kSt * kStB + (threadIdx.x >> 5) * kOutWarpBytes;
    // per-pattern partial results of the two category halves: [5][2][128]
    // floats at the start of the staging area (idle until the stores of pass 2)
    float* xch = reinterpret_cast<float*>(stages + kSt * kStB);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;      // bit 0 empty, 1 full, 2 done wait gave up
    __shared__ unsigned produced_sh, consumed_sh;
    __shared__ float red[8];
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
        for (int s = 0; s < kSt; ++s) {
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
    unsigned pairs_done = 0;   // (operand, category) products issued by this CTA
    unsigned items_done = 0;   // items with at least one product

    const int n_items = n_ops * a.n_tiles;
    // thread 0: pairs loaded and pairs multiplied so far (both absolute)
    unsigned produced_c = 0, consumed_c = 0;
    // Load pair i of an item (operand c, category r) into stage g % kSt once
    // the products that last read it are done; false if that wait gave up.
    auto produce = [&](const TcOp& o, int q0, int i, unsigned g) -> bool {
        const int s = g % kSt;
        if (!mbar_wait(&empty[s], ((g / kSt) & 1) ^ 1)) {
            abort_sh |= 1;
            return false;
        }
        const bool m0 = o.kind[0] == kInternal || o.kind[0] == kTipPartials;
        const int c = m0 ? (i < R ? 0 : 1) : 1;
        const int r = i % R;
        unsigned char* st = stages + s * kStB;
        mbar_expect_tx(&full[s], TcPipe<SPLIT, SPLITA>::tx_bytes);
        const int arow = (o.child[c] * R + r) * a.Ppad + q0;
        const int brow = o.brow[c] + r * kTcN;
        const CUtensorMap* am = o.kind[c] == kTipPartials ? &tm_tip : &tm_part;
        tma_load_2d(st, am, 0, arow, &full[s]);
        tma_load_2d(st + kAChunk, am, 32, arow, &full[s]);
        tma_load_2d(st + kBOff, &tm_mat, 0, brow, &full[s]);
        tma_load_2d(st + kBOff + kBChunk, &tm_mat, 32, brow, &full[s]);
        if (SPLIT) {
            const int lrow = brow + 2 * R * kTcN;
            tma_load_2d(st + kBOff + 2 * kBChunk, &tm_mat, 0, lrow, &full[s]);
            tma_load_2d(st + kBOff + 3 * kBChunk, &tm_mat, 32, lrow, &full[s]);
        }
        return true;
    };
    // the k-steps of one (operand, category) product from stage st into d
    auto issue_products = [&](unsigned char* st, uint32_t d) {
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
            const int chunk = ks >> 2, kin = (ks & 3) * 32;
            const uint64_t ad = sw128_desc(st + chunk * kAChunk + kin);
            const uint64_t bd = sw128_desc(st + kBOff + chunk * kBChunk + kin);
            mma_tf32(d, ad, bd, ks > 0 ? 1u : 0u);
            if (SPLIT) {
                const uint64_t bl = sw128_desc(st + kBOff + (2 + chunk) * kBChunk + kin);
                mma_tf32(d, ad, bl, 1u);
            }
            if (SPLITA) {
                const uint64_t al = sw128_desc(st + (2 + chunk) * kAChunk + kin);
                mma_tf32(d, al, bd, 1u);
            }
        }
    };
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int k = item / a.n_tiles, tile = item % a.n_tiles;
        const TcOp op = ops[k];
        const int p0 = tile * kTcM;
        const bool mma[2] = {op.kind[0] == kInternal || op.kind[0] == kTipPartials,
                             op.kind[1] == kInternal || op.kind[1] == kTipPartials};
        const int n_pairs = (mma[0] + mma[1]) * R;
        if constexpr (SPLITA) {
            // every thread takes part in each pair: wait for its copy, split
            // A, then thread 0 issues the products
            bool ok = true;
            for (int j = 0; j < n_pairs && ok; ++j) {
                const unsigned g = pairs_done + (unsigned)j;
                if (tid == 0) {
                    while (ok && produced_c < pairs_done + n_pairs && produced_c < g + kSt) {
                        ok = produce(op, p0, (int)(produced_c - pairs_done), produced_c);
                        produced_c += ok;
                    }
                }
                const int s = g % kSt;
                bool got = true;
                if (ok) got = mbar_wait(&full[s], (g / kSt) & 1);
                if (tid == 0 && !ok) got = false;
                if (!got) atomicOr(&abort_sh, 2);
                if (__syncthreads_or(!got)) {
                    ok = false;
                    break;
                }
                unsigned char* st = stages + s * kStB;
                float4* A4 = reinterpret_cast<float4*>(st);
                float4* L4 = reinterpret_cast<float4*>(st + 2 * kAChunk);
#pragma unroll 4
                for (int i = tid; i < 2 * kAChunk / 16; i += kTcThreads) {
                    const float4 v = A4[i];
                    float4 h, l;
                    h.x = tf32_trunc(v.x);
                    h.y = tf32_trunc(v.y);
                    h.z = tf32_trunc(v.z);
                    h.w = tf32_trunc(v.w);
                    l.x = tf32_trunc(v.x - h.x);
                    l.y = tf32_trunc(v.y - h.y);
                    l.z = tf32_trunc(v.z - h.z);
                    l.w = tf32_trunc(v.w - h.w);
                    A4[i] = h;
                    L4[i] = l;
                }
                fence_proxy_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const int c = mma[0] ? (j < R ? 0 : 1) : 1;
                    const int r = j % R;
                    issue_products(st, tmem + (uint32_t)(r * 2 * kTcN + c * kTcN));
                    mma_commit(&empty[s]);
                    consumed_c = g + 1;
                }
            }
            if (tid == 0) {
                if (ok && n_pairs > 0) mma_commit(&done);
                const int nxt = item + gridDim.x;
                if (ok && nxt < n_items) {
                    const TcOp opn = ops[nxt / a.n_tiles];
                    const int p0n = (nxt % a.n_tiles) * kTcM;
                    const bool mn0 = opn.kind[0] == kInternal || opn.kind[0] == kTipPartials;
                    const bool mn1 = opn.kind[1] == kInternal || opn.kind[1] == kTipPartials;
                    const unsigned base = pairs_done + n_pairs;
                    const unsigned pn = (unsigned)((mn0 + mn1) * R);
                    while (ok && produced_c < base + pn && produced_c < base + kSt) {
                        ok = produce(opn, p0n, (int)(produced_c - base), produced_c);
                        produced_c += ok;
                    }
                }
                produced_sh = produced_c;
                consumed_sh = consumed_c;
            }
        } else if (tid == 0) {
            // Pairs are numbered across the CTA's items: pair g uses stage
            // g % kSt. Up to kSt pairs are loaded ahead of the products; the
            // first pairs of the next item are loaded before this item's
            // epilogue, so their copies overlap it.
            bool ok = true;
            while (ok && n_pairs > 0 && consumed_c < pairs_done + n_pairs) {
                while (ok && produced_c < pairs_done + n_pairs && produced_c < consumed_c + kSt) {
                    ok = produce(op, p0, (int)(produced_c - pairs_done), produced_c);
                    produced_c += ok;
                }
                if (!ok) break;
                const unsigned g = consumed_c;
                const int s = g % kSt;
                ok = mbar_wait(&full[s], (g / kSt) & 1);
                if (!ok) {
                    abort_sh |= 2;
                    break;
                }
                tc_fence_after();
                const int j = (int)(g - pairs_done);
                const int c = mma[0] ? (j < R ? 0 : 1) : 1;
                const int r = j % R;
                issue_products(stages + s * kStB, tmem + (uint32_t)(r * 2 * kTcN + c * kTcN));
                mma_commit(&empty[s]);
                ++consumed_c;
            }
            if (n_pairs > 0) mma_commit(&done);
            // the next item's first pairs
            const int nxt = item + gridDim.x;
            if (ok && nxt < n_items) {
                const TcOp opn = ops[nxt / a.n_tiles];
                const int p0n = (nxt % a.n_tiles) * kTcM;
                const bool mn0 = opn.kind[0] == kInternal || opn.kind[0] == kTipPartials;
                const bool mn1 = opn.kind[1] == kInternal || opn.kind[1] == kTipPartials;
                const unsigned base = pairs_done + n_pairs;
                const unsigned pn = (unsigned)((mn0 + mn1) * R);
                while (ok && produced_c < base + pn && produced_c < base + kSt) {
                    ok = produce(opn, p0n, (int)(produced_c - base), produced_c);
                    produced_c += ok;
                }
            }
            produced_sh = produced_c;
            consumed_sh = consumed_c;
        }
        __syncthreads();
        bool fail = abort_sh != 0;
        if (!fail && n_pairs > 0 && !mbar_wait(&done, items_done & 1)) {
            fail = true;
            atomicOr(&abort_sh, 4);
        }
        if (__syncthreads_or(fail)) break;
        if (n_pairs > 0) {
            tc_fence_after();
            ++items_done;
        }
        pairs_done += n_pairs;

        // ---- epilogue: lane (tid & 127) <-> pattern p0 + (tid & 127); warp
        // half hf takes categories [rb, re) ----------------------------------
        const int pl = tid & 127, hf = warp >> 2;
        const int p = p0 + pl;
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const int rb = hf ? (R + 1) / 2 : 0, re = hf ? R : (R + 1) / 2;
        // partial k of this half into the exchange area, then (after a
        // barrier) both halves' values of this pattern
        auto put_x = [&](int k, float v) { xch[(k * 2 + hf) * 128 + pl] = v; };
        auto get_x = [&](int k, int h) { return xch[(k * 2 + h) * 128 + pl]; };
        int sidx[2] = {0, 0};
        bool amb[2] = {false, false};
        for (int c = 0; c < 2; ++c)
            if (op.kind[c] == kTipStates) {
                const int s = a.tips[(size_t)op.child[c] * a.Ppad + p];
                amb[c] = !(s >= 0 && s < a.S);
                sidx[c] = s;
            }
        // all 64 values (category r) of operand c: its accumulator columns,
        // or the tip's P^T row (+ the lo row with split matrices), or the row
        // sums of P for an ambiguous code; the row loads are issued together
        auto operand64 = [&](int c, int r, float* v) {
            if (mma[c]) {
                tmem_ld64(lane_base + (uint32_t)(r * 2 * kTcN + c * kTcN), v);
                return;
            }
            const int slot_base = op.look[c];
            const float* src =
                amb[c] ? a.rowsum + (size_t)(slot_base / ((SPLIT ? 4 : 2) * R * kTcN * kTcN)) * R * kTcN +
                             (size_t)r * kTcN
                       : a.matw + (size_t)slot_base + (size_t)r * kTcN * kTcN + (size_t)sidx[c] * kTcN;
            const float4* s4 = reinterpret_cast<const float4*>(src);
            float4 f[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) f[u] = __ldg(s4 + u);
            if (SPLIT && !amb[c]) {
                const float4* l4 = reinterpret_cast<const float4*>(src + kLoFloats);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float4 l = __ldg(l4 + u);
                    f[u].x += l.x;
                    f[u].y += l.y;
                    f[u].z += l.z;
                    f[u].w += l.w;
                }
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                v[4 * u] = f[u].x;
                v[4 * u + 1] = f[u].y;
                v[4 * u + 2] = f[u].z;
                v[4 * u + 3] = f[u].w;
            }
        };
        auto qvals64 = [&](int r, float* v) {  // parent pre-order partial (pre1), category r
            if (op.qin < 0) {
#pragma unroll
                for (int i = 0; i < 64; ++i) v[i] = (float)a.pi[i];
            } else {
                const float4* s4 = reinterpret_cast<const float4*>(
                    a.pool + (size_t)op.qin * a.bstride + ((size_t)r * a.Ppad + p) * kTcN);
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
        };
        auto scale_of = [](float m, float* f1, float* f2) -> int {
            const int e = frexp_exp_f(m);
            *f1 = 1.f;
            *f2 = 1.f;
            if (e != 0) {
                const int kk = -e;
                if (kk >= -126 && kk <= 126) *f1 = pow2f(kk);
                else {
                    *f1 = pow2f(kk / 2);
                    *f2 = pow2f(kk - kk / 2);
                }
            }
            return e;
        };
        // stored partials: TF32-rounded (the tensor core reads them exactly),
        // or full FP32 when A is split on chip
        auto rnd = [](float x) { return SPLITA ? x : to_tf32(x); };
        // A 64-float row per thread (pattern), scaled and rounded, stored
        // through the warp's staging area: half rows written with their
        // 16-byte units XOR-swizzled by the row, read back four half rows
        // per instruction and stored as whole cache lines (a plain store of
        // one row per thread touches 32 lines per instruction).
        // tile_base: row 0 of this warp's 32 patterns (row stride 64 floats).
        auto store_row = [&](float* tile_base, const float* v, float f1, float f2) {
            const int ln = tid & 31;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int i = h * 32 + 4 * j;
                    *reinterpret_cast<float4*>(wout + ln * 128 + ((j ^ (ln & 7)) << 4)) =
                        make_float4(rnd(v[i] * f1 * f2), rnd(v[i + 1] * f1 * f2),
                                    rnd(v[i + 2] * f1 * f2), rnd(v[i + 3] * f1 * f2));
                }
                __syncwarp();
                const int u = ln & 7;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + (ln >> 3);
                    const float4 f =
                        *reinterpret_cast<const float4*>(wout + rr * 128 + ((u ^ (rr & 7)) << 4));
                    *reinterpret_cast<float4*>(tile_base + (size_t)rr * kTcN + h * 32 + 4 * u) = f;
                }
                __syncwarp();
            }
        };
        const size_t wrow0 = (size_t)(p0 + (warp & 3) * 32) * kTcN;   // this warp's first row
        const bool real = p < a.Ppad;  // always true (tiles cover Ppad)
        const float wp = (p < a.Ppad) ? (float)a.patw[p] : 0.f;

        if (MODE == kPost) {
            int cum = 0;
            for (int c = 0; c < 2; ++c)
                if (op.kind[c] == kInternal) cum += a.epool[(size_t)op.child[c] * a.Ppad + p];
            // pass 1: the products of all categories and their maximum; each
            // category's products replace operand 0's accumulator in TMEM
            float m = 0.f;
            for (int r = rb; r < re; ++r) {
                float x[64], y[64];
                operand64(0, r, x);
                operand64(1, r, y);
#pragma unroll
                for (int i = 0; i < 64; ++i) {
                    x[i] *= y[i];
                    m = fmaxf(m, x[i]);
                }
                tmem_st64(lane_base + (uint32_t)(r * 2 * kTcN), x);
            }
            put_x(0, m);
            __syncthreads();
            m = fmaxf(get_x(0, 0), get_x(0, 1));
            __syncthreads();   // the exchange area is the stores' staging area
            float f1 = 1.f, f2 = 1.f;
            if (a.rescale) cum += post_scale(m, &f1, &f2);
            // pass 2: rescale, round to TF32, store
            float* dst = a.pool + (size_t)op.dest * a.bstride + wrow0;
            for (int r = rb; r < re; ++r) {
                float z[64];
                tmem_ld64(lane_base + (uint32_t)(r * 2 * kTcN), z);
                store_row(dst + (size_t)r * a.Ppad * kTcN, z, f1, f2);
            }
            if (hf == 0) a.epool[(size_t)op.dest * a.Ppad + p] = cum;
        } else if (MODE == kPre1) {
            // pass 1 over categories: den, the maxima of u_a = q o v_b and
            // u_b = q o v_a, tip numerators u_c . dP_c[:, s]; u of internal
            // children replaces their accumulators in TMEM
            float den = 0.f, mu[2] = {0.f, 0.f}, num[2] = {0.f, 0.f};
            const bool tipg[2] = {op.kind[0] == kTipStates && op.edge[0] >= 0,
                                  op.kind[1] == kTipStates && op.edge[1] >= 0};
            for (int r = rb; r < re; ++r) {
                float x[64], y[64];
                operand64(0, r, x);
                operand64(1, r, y);
                float dr = 0.f;
                {
                    float z[64];
                    qvals64(r, z);
#pragma unroll
                    for (int i = 0; i < 64; ++i) {
                        const float va = x[i], vb = y[i];
                        dr += z[i] * va * vb;
                        x[i] = z[i] * vb;  // u_a
                        y[i] = z[i] * va;  // u_b
                        mu[0] = fmaxf(mu[0], x[i]);
                        mu[1] = fmaxf(mu[1], y[i]);
                    }
                }
                den += a.catw[r] * dr;
                for (int c = 0; c < 2; ++c) {
                    if (!tipg[c]) continue;
                    // u_c . (a row of dP^T); an ambiguous code gives the row
                    // sums of dP, which are zero
                    const int srow = amb[c] ? 0 : sidx[c];
                    const float4* d4 = reinterpret_cast<const float4*>(
                        a.matw + (size_t)op.dlook[c] + (size_t)r * kTcN * kTcN + (size_t)srow * kTcN);
                    const float* uc = c == 0 ? x : y;
                    float nr = 0.f;
#pragma unroll
                    for (int g4 = 0; g4 < 4; ++g4) {
                        float4 f[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) f[u] = __ldg(d4 + 4 * g4 + u);
                        if (SPLIT) {
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const float4 l = __ldg(d4 + 4 * g4 + u + kLoFloats / 4);
                                f[u].x += l.x;
                                f[u].y += l.y;
                                f[u].z += l.z;
                                f[u].w += l.w;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int b = 16 * g4 + 4 * u;
                            nr += uc[b] * f[u].x + uc[b + 1] * f[u].y + uc[b + 2] * f[u].z +
                                  uc[b + 3] * f[u].w;
                        }
                    }
                    num[c] += a.catw[r] * nr;
                }
                if (op.uout[0] >= 0) tmem_st64(lane_base + (uint32_t)(r * 2 * kTcN), x);
                if (op.uout[1] >= 0) tmem_st64(lane_base + (uint32_t)(r * 2 * kTcN + kTcN), y);
            }
            put_x(0, den);
            put_x(1, mu[0]);
            put_x(2, mu[1]);
            put_x(3, num[0]);
            put_x(4, num[1]);
            __syncthreads();
            den = get_x(0, 0) + get_x(0, 1);
            mu[0] = fmaxf(get_x(1, 0), get_x(1, 1));
            mu[1] = fmaxf(get_x(2, 0), get_x(2, 1));
            num[0] = get_x(3, 0) + get_x(3, 1);
            num[1] = get_x(4, 0) + get_x(4, 1);
            __syncthreads();
            for (int c = 0; c < 2; ++c) {
                if (!tipg[c]) continue;
                const float g =
                    block_sum256(hf == 0 ? wp * ((amb[c] ? 0.f : num[c]) / den) : 0.f, red);
                if (tid == 0) a.gpart[(size_t)op.edge[c] * a.n_tiles + tile] = (double)g;
            }
            // pass 2: each internal child's u, rescaled, to its pre buffer;
            // its ratio denominator carries the same scale as u
            for (int c = 0; c < 2; ++c) {
                if (op.uout[c] < 0) continue;
                float f1, f2;
                const int e = scale_of(mu[c], &f1, &f2);
                float* dst = a.pool + (size_t)op.uout[c] * a.bstride + wrow0;
                for (int r = rb; r < re; ++r) {
                    float u[64];
                    tmem_ld64(lane_base + (uint32_t)(r * 2 * kTcN + c * kTcN), u);
                    store_row(dst + (size_t)r * a.Ppad * kTcN, u, f1, f2);
                }
                float d = den;
                if (e != 0) d = (-e >= -126 && -e <= 126) ? den * pow2f(-e)
                                                         : den * pow2f(-e / 2) * pow2f(-e - (-e / 2));
                if (hf == 0) a.epool[(size_t)op.uout[c] * a.Ppad + p] = __float_as_int(d);
            }
        } else {  // kPre2: operand 0 = q_c = u_c P_c (B = P^T), operand 1 = Q x_c
                  // (or dP x_c for a general derivative, paired with u_c)
            const float den = __int_as_float(a.epool[(size_t)op.dest * a.Ppad + p]);
            const float* ub = a.pool + (size_t)op.dest * a.bstride + (size_t)p * kTcN;
            float num = 0.f, m = 0.f;
            for (int r = rb; r < re; ++r) {
                float x[64], y[64];
                tmem_ld64(lane_base + (uint32_t)(r * 2 * kTcN), x);
                tmem_ld64(lane_base + (uint32_t)(r * 2 * kTcN + kTcN), y);
                float nr = 0.f;
                if (a.dgen) {
                    const float4* u4 = reinterpret_cast<const float4*>(ub + (size_t)r * a.Ppad * kTcN);
                    float4 f[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) f[u] = u4[u];
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        nr += f[u].x * y[4 * u] + f[u].y * y[4 * u + 1] + f[u].z * y[4 * u + 2] +
                              f[u].w * y[4 * u + 3];
                } else {
#pragma unroll
                    for (int i = 0; i < 64; ++i) nr += x[i] * y[i];
                }
#pragma unroll
                for (int i = 0; i < 64; ++i) m = fmaxf(m, x[i]);
                num += a.catw[r] * (a.dgen ? 1.f : a.rates[r]) * nr;
            }
            put_x(0, num);
            put_x(1, m);
            __syncthreads();
            num = get_x(0, 0) + get_x(0, 1);
            m = fmaxf(get_x(1, 0), get_x(1, 1));
            __syncthreads();
            if (op.edge[0] >= 0) {
                const float g = block_sum256(hf == 0 ? wp * (num / den) : 0.f, red);
                if (tid == 0) a.gpart[(size_t)op.edge[0] * a.n_tiles + tile] = (double)g;
            }
            float f1, f2;
            scale_of(m, &f1, &f2);
            float* dst = a.pool + (size_t)op.dest * a.bstride + wrow0;
            for (int r = rb; r < re; ++r) {
                float x[64];
                tmem_ld64(lane_base + (uint32_t)(r * 2 * kTcN), x);
                store_row(dst + (size_t)r * a.Ppad * kTcN, x, f1, f2);
            }
        }
        (void)real;
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (abort_sh && tid == 0) {
        // where the wait gave up (bits 0-2) and in which kernel mode (bits 8+)
        atomicOr(a.err, abort_sh | (1 << (8 + MODE)));
        // bounded drain of copies and products still in flight
        for (unsigned g = consumed_sh; g < produced_sh; ++g)
            mbar_wait(&full[g % kSt], (g / kSt) & 1);
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
                          const double* __restrict__ catw, int* __restrict__ numeric_err) {
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
            if (!(L > 0.0) || !isfinite(l)) atomicOr(numeric_err, 1);
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
    a.patw = I->d_patw;
    a.pi = nullptr;
    a.gpart = nullptr;
    a.dgen = 0;
    a.R = I->R;
    a.Ppad = I->Ppad;
    a.S = I->S;
    a.n_tiles = I->Ppad / kTcM;
    a.rescale = I->rescale;
    a.bstride = (size_t)I->R * I->Ppad * kTcN;
    a.err = I->d_err + 2;
    for (int r = 0; r < kMaxCat; ++r) {
        a.catw[r] = (float)(r < I->R ? I->h_catw[r] : 0.0);
        a.rates[r] = (float)(r < I->R ? I->h_rates[r] : 0.0);
    }
    return a;
}

// Row of the P (which = 0) or P^T (which = 1) block of a slot in the matrix
// map, category 0; float offset of the same block in the matrix array.
// A slot holds 2 blocks of R 64 x 64 floats (P, P^T), 4 with split matrices
// (P_hi, P_hi^T, P_lo, P_lo^T); a model's Q copy 1 block, or 4 (Q_hi, -,
// Q_lo, -) so that lo is always two blocks after hi.
int blocks_per_slot(const Instance* I) { return I->split ? 4 : 2; }
int blocks_per_q(const Instance* I) { return I->split ? 4 : 1; }
int brow_of(const Instance* I, int slot, int which) {
    return (slot * blocks_per_slot(I) + which) * I->R * kTcN;
}
int look_of(const Instance* I, int slot, int which) {
    return (int)((size_t)slot * I->matw_stride + (size_t)which * I->R * kTcN * kTcN);
}
int qrow_of(const Instance* I, int model) {
    return (I->n_mats * blocks_per_slot(I) + model * blocks_per_q(I)) * I->R * kTcN;
}

// Q in TF32 for every category block; with split matrices also the lo
// term (the TF32 truncation of fl32(Q) - Q_hi) two blocks later.
__global__ void k_q_tc(const double* __restrict__ Q, float* __restrict__ dst, int R, int split) {
    for (int idx = threadIdx.x; idx < R * kTcN * kTcN; idx += blockDim.x) {
        const float f = (float)Q[idx % (kTcN * kTcN)];
        const float hi = to_tf32(f);
        dst[idx] = hi;
        if (split)
            dst[idx + (size_t)2 * R * kTcN * kTcN] =
                __uint_as_float(__float_as_uint(f - hi) & 0xffffe000u);
    }
}

template <int MODE, bool SPLIT, bool SPLITA>
void launch_mode_t(Instance* I, const TcOp* d, int n, TcArgs a) {
    const size_t smem = (size_t)TcPipe<SPLIT, SPLITA>::stages * TcPipe<SPLIT, SPLITA>::bytes +
                        (kTcThreads / 32) * kOutWarpBytes + 1024;
    cudaFuncSetAttribute(k_tc<MODE, SPLIT, SPLITA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int sms = 0, dev_id = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(I->tmaps.data());
    const int items = n * a.n_tiles;
    const int grid = std::max(1, std::min(items, sms));
    k_tc<MODE, SPLIT, SPLITA><<<grid, kTcThreads, smem, I->stream>>>(m[0], m[1], m[2], d, n, a);
    I->launches += 1;
}

template <int MODE>
void launch_mode(Instance* I, const TcOp* d, int n, TcArgs a) {
    if (I->split_partials) launch_mode_t<MODE, true, true>(I, d, n, a);
    else if (I->split) launch_mode_t<MODE, true, false>(I, d, n, a);
    else launch_mode_t<MODE, false, false>(I, d, n, a);
}

void tc_operand(const Instance* I, TcOp& t, int c, int buf, int slot) {
    if (buf < I->n_tips) {
        t.kind[c] = I->tip_set[buf] == 1 ? kTipStates : kTipPartials;
        t.child[c] = buf;
    } else {
        t.kind[c] = kInternal;
        t.child[c] = buf - I->n_tips;
    }
    t.brow[c] = brow_of(I, slot, 0);
    t.look[c] = look_of(I, slot, 1);
}

// ---------------------------------------------------------------------------
// On-chip subtree-fused post-order (TF32 storage, plain or split matrices)
// ---------------------------------------------------------------------------
// One CTA walks the whole op list for one 128-pattern tile at a time (ops in
// a depth-first post-order from the host), instead of one launch per tree
// level. The result of each op stays in tensor memory as the A operand of
// the next op (TMEM columns [0, 256): 4 categories x 64 states, TF32
// values), so a child produced by the op just before is never read back
// from HBM: it is multiplied in place (tcgen05.mma with A in TMEM). Other
// children come from HBM through TMA as before; tips with states are
// lookups. Every op's result is also stored, as by the level-by-level
// kernel (same values: same products, same accumulation order, same
// rescaling), so the pre-order pass and later calls can read any buffer.
//
// Roles (warp-specialised, 192 threads):
//   warp 0  TMA: A tiles of children read from HBM and B tiles (P, P_lo),
//           a ring of kSt stages (full / empty mbarriers);
//   warp 1  TMEM owner and MMA issuer: per (op, category) the products of
//           both children into one of two accumulator buffers (columns
//           256 + 128 b, child c at + 64 c), committed to acc_full[b];
//   warps 2-5  epilogue, one TMEM lane (pattern) per thread: pass 1 per
//           category multiplies the children (or a tip's P^T row), takes
//           the maximum, releases the accumulator buffer (acc_empty[b]) and
//           parks the unscaled product in the category's A columns; pass 2
//           rescales by the power of two of the maximum over categories,
//           rounds to TF32, rewrites the A columns and stores the partials
//           and exponents; then each warp publishes the op as done (a
//           counter per warp, release / acquire ordering), which the MMA
//           warp waits for before it multiplies an op's on-chip child.
// Every wait is bounded by elapsed time and by an abort flag, so a wait
// that gives up stops all roles; the kernel then drains its copies and
// products and frees TMEM.
struct __align__(16) FuseOp {
    int child[2];
    int kind[2];      // kInternal, kTipPartials: MMA; kTipStates: lookup
    int brow[2];      // matrix-map row of P, category 0
    int look[2];      // float offset of P^T, category 0 (tip lookups)
    int dest;         // output buffer (pool index)
    int prev;         // the child (0, 1) that is the previous op's result; -1 none
    int src[2];       // op of this list that stores child c (read from HBM); -1 none
    int tbrow[2];     // matrix-map row of P^T, category 0 (tip lookups from shared memory)
    int pad[2];
};
static_assert(sizeof(FuseOp) == kTcOpBytes, "fused descriptor size");

constexpr int kFuseThreads = 192;
constexpr int kPrevCols = 256;   // TMEM columns of the on-chip result

// MMA stages (A, B, B_lo), then a two-slot ring of P^T blocks (P^T_lo)
// for the epilogue's tip lookups.
template <bool SPLIT>
struct FusePipe {
    static constexpr int stages = SPLIT ? 2 : 3;
    static constexpr int bytes = 2 * kAChunk + (SPLIT ? 4 : 2) * kBChunk;
    static constexpr int tip_slots = 2;
    static constexpr int tip_bytes = (SPLIT ? 4 : 2) * kBChunk;
    static constexpr int out_bytes = 4 * 32 * 128;   // per epilogue warp: 32 half rows
    static constexpr size_t smem =
        (size_t)stages * bytes + (size_t)tip_slots * tip_bytes + out_bytes;
};

template <bool SPLIT>
__global__ void __launch_bounds__(kFuseThreads, 1)
k_tc_fused(const __grid_constant__ CUtensorMap tm_part, const __grid_constant__ CUtensorMap tm_tip,
           const __grid_constant__ CUtensorMap tm_mat, const FuseOp* __restrict__ ops, int n_ops,
           TcArgs a) {
    constexpr int kSt = FusePipe<SPLIT>::stages;
    constexpr int kStB = FusePipe<SPLIT>::bytes;
    constexpr int kBOff = 2 * kAChunk;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    unsigned char* stages = smem_tc + ((1024u - (smem_u32(smem_tc) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], acc_full[2], acc_empty[2],
        tip_full[2], tip_empty[2], done;
    unsigned char* tip_area = stages + kSt * kStB;
    unsigned char* out_area = tip_area + FusePipe<SPLIT>::tip_slots * FusePipe<SPLIT>::tip_bytes;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;  // bit 0 empty, 1 full, 2 acc_empty, 3 acc_full, 4/6 op done
    __shared__ unsigned ready_sh[4];  // ops each epilogue warp has finished
    __shared__ unsigned loads_sh, used_sh, tip_loads_sh, tip_used_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_v = &abort_sh;

    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                smem_u32(&tmem_base_sh)),
            "r"(kTmemCols)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kSt; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);   // one arrival per epilogue warp
            mbar_init(&tip_full[b], 1);
            mbar_init(&tip_empty[b], 4);
        }
        mbar_init(&done, 1);
        abort_sh = 0;
        for (int w = 0; w < 4; ++w) ready_sh[w] = 0;
        loads_sh = used_sh = tip_loads_sh = tip_used_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int R = a.R;
    auto on_mma = [](const FuseOp& o, int c) {
        return o.kind[c] == kInternal || o.kind[c] == kTipPartials;
    };

    if (warp == 0) {
        // ---- TMA producer ----------------------------------------------------
        if (lane == 0) {
            unsigned g = 0, gt = 0, base = 0;   // base: ops of earlier tiles
            for (int tile = blockIdx.x; tile < a.n_tiles && !*abort_v; tile += gridDim.x,
                     base += (unsigned)n_ops) {
                const int q0 = tile * kTcM;
                for (int k = 0; k < n_ops && !*abort_v; ++k) {
                    const FuseOp o = ops[k];
                    // a child this launch stores is read only after the
                    // epilogue of the op that stores it is done with it
                    for (int c = 0; c < 2; ++c) {
                        if (o.src[c] < 0 || o.prev == c) continue;
                        const unsigned need = base + (unsigned)o.src[c] + 1;
                        const unsigned long long t0 = global_ns();
                        for (int w = 0; w < 4 && !*abort_v; ++w)
                            while (ld_acquire_cta(&ready_sh[w]) < need) {
                                if (*abort_v || global_ns() - t0 > kWaitNs) {
                                    atomicOr(&abort_sh, 64);
                                    break;
                                }
                            }
                        fence_proxy_async_global();
                    }
                    for (int r = 0; r < R && !*abort_v; ++r)
                        for (int c = 0; c < 2; ++c) {
                            if (o.kind[c] == kTipStates) {
                                // the P^T block (and its lo block) of the tip's
                                // edge for the epilogue's row lookups
                                const int ts = gt % 2;
                                if (!mbar_wait_or_abort(&tip_empty[ts], ((gt / 2) & 1) ^ 1, abort_v)) {
                                    atomicOr(&abort_sh, 1);
                                    break;
                                }
                                unsigned char* tb = tip_area + ts * FusePipe<SPLIT>::tip_bytes;
                                mbar_expect_tx(&tip_full[ts], FusePipe<SPLIT>::tip_bytes);
                                const int trow = o.tbrow[c] + r * kTcN;
                                tma_load_2d(tb, &tm_mat, 0, trow, &tip_full[ts]);
                                tma_load_2d(tb + kBChunk, &tm_mat, 32, trow, &tip_full[ts]);
                                if (SPLIT) {
                                    const int lrow = trow + 2 * R * kTcN;
                                    tma_load_2d(tb + 2 * kBChunk, &tm_mat, 0, lrow, &tip_full[ts]);
                                    tma_load_2d(tb + 3 * kBChunk, &tm_mat, 32, lrow, &tip_full[ts]);
                                }
                                ++gt;
                                continue;
                            }
                            if (!on_mma(o, c)) continue;
                            const int s = g % kSt;
                            if (!mbar_wait_or_abort(&empty[s], ((g / kSt) & 1) ^ 1, abort_v)) {
                                atomicOr(&abort_sh, 1);
                                break;
                            }
                            unsigned char* st = stages + s * kStB;
                            const bool fromA = o.prev != c;
                            mbar_expect_tx(&full[s],
                                           (fromA ? 2 * kAChunk : 0) + (SPLIT ? 4 : 2) * kBChunk);
                            if (fromA) {
                                const int arow = (o.child[c] * R + r) * a.Ppad + q0;
                                const CUtensorMap* am = o.kind[c] == kTipPartials ? &tm_tip : &tm_part;
                                tma_load_2d(st, am, 0, arow, &full[s]);
                                tma_load_2d(st + kAChunk, am, 32, arow, &full[s]);
                            }
                            const int brow = o.brow[c] + r * kTcN;
                            tma_load_2d(st + kBOff, &tm_mat, 0, brow, &full[s]);
                            tma_load_2d(st + kBOff + kBChunk, &tm_mat, 32, brow, &full[s]);
                            if (SPLIT) {
                                const int lrow = brow + 2 * R * kTcN;
                                tma_load_2d(st + kBOff + 2 * kBChunk, &tm_mat, 0, lrow, &full[s]);
                                tma_load_2d(st + kBOff + 3 * kBChunk, &tm_mat, 32, lrow, &full[s]);
                            }
                            ++g;
                        }
                }
            }
            loads_sh = g;
            tip_loads_sh = gt;
        }
    } else if (warp == 1) {
        // ---- MMA issuer ------------------------------------------------------
        if (lane == 0) {
            unsigned g = 0, cat = 0, nop = 0;
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < a.n_tiles; tile += gridDim.x) {
                for (int k = 0; ok && k < n_ops; ++k, ++nop) {
                    const FuseOp o = ops[k];
                    if (o.prev >= 0) {
                        // the previous op's result must be complete in TMEM
                        const unsigned long long t0 = global_ns();
                        for (int w = 0; ok && w < 4; ++w)
                            while (ld_acquire_cta(&ready_sh[w]) < nop) {
                                if (*abort_v || global_ns() - t0 > kWaitNs) {
                                    ok = false;
                                    atomicOr(&abort_sh, 16);
                                    break;
                                }
                            }
                        if (!ok) break;
                        tc_fence_after();
                    }
                    for (int r = 0; ok && r < R; ++r, ++cat) {
                        const int b = cat & 1;
                        if (!mbar_wait_or_abort(&acc_empty[b], ((cat >> 1) & 1) ^ 1, abort_v)) {
                            ok = false;
                            atomicOr(&abort_sh, 4);
                            break;
                        }
                        tc_fence_after();
                        for (int c = 0; c < 2; ++c) {
                            if (!on_mma(o, c)) continue;
                            const int s = g % kSt;
                            if (!mbar_wait_or_abort(&full[s], (g / kSt) & 1, abort_v)) {
                                ok = false;
                                atomicOr(&abort_sh, 2);
                                break;
                            }
                            tc_fence_after();
                            const uint32_t d = tmem + (uint32_t)(kPrevCols + b * 2 * kTcN + c * kTcN);
                            unsigned char* st = stages + s * kStB;
#pragma unroll
                            for (int ks = 0; ks < 8; ++ks) {
                                const int chunk = ks >> 2, kin = (ks & 3) * 32;
                                const uint64_t bd = sw128_desc(st + kBOff + chunk * kBChunk + kin);
                                const uint64_t bl = sw128_desc(st + kBOff + (2 + chunk) * kBChunk + kin);
                                if (o.prev == c) {
                                    const uint32_t at = tmem + (uint32_t)(r * kTcN + ks * 8);
                                    mma_tf32_ta(d, at, bd, ks > 0 ? 1u : 0u);
                                    if (SPLIT) mma_tf32_ta(d, at, bl, 1u);
                                } else {
                                    const uint64_t ad = sw128_desc(st + chunk * kAChunk + kin);
                                    mma_tf32(d, ad, bd, ks > 0 ? 1u : 0u);
                                    if (SPLIT) mma_tf32(d, ad, bl, 1u);
                                }
                            }
                            mma_commit(&empty[s]);
                            ++g;
                        }
                        if (!ok) break;
                        mma_commit(&acc_full[b]);
                    }
                }
            }
            used_sh = g;
            // every product issued has finished before TMEM is released
            mma_commit(&done);
            if (!mbar_wait(&done, 0)) atomicOr(&abort_sh, 32);
        }
    } else {
        // ---- epilogue: thread <-> TMEM lane 32 (warp % 4) + lane -----------
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
        unsigned cat = 0, nop = 0;
        bool ok = true;
        // Stores go out through a per-warp shared-memory transpose: each
        // thread holds one pattern's row (256 bytes), and a store of the
        // rows as they are would touch 32 cache lines per instruction. Half
        // rows (128 bytes) are written with the 16-byte units XOR-swizzled by
        // the row (j ^ (row & 7): 4-way conflicts instead of 32), read back
        // four whole half rows per instruction and stored as full lines.
        unsigned char* wout = out_area + quarter * 32 * 128;
        auto store_row = [&](float* tile_base, const float* z) {
            // tile_base: row 0 of this warp's 32 rows (row stride 64 floats)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    *reinterpret_cast<float4*>(wout + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                        make_float4(z[h * 32 + 4 * j], z[h * 32 + 4 * j + 1], z[h * 32 + 4 * j + 2],
                                    z[h * 32 + 4 * j + 3]);
                __syncwarp();
                const int u = lane & 7;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + (lane >> 3);
                    const float4 f =
                        *reinterpret_cast<const float4*>(wout + rr * 128 + ((u ^ (rr & 7)) << 4));
                    *reinterpret_cast<float4*>(tile_base + (size_t)rr * kTcN + h * 32 + 4 * u) = f;
                }
                __syncwarp();
            }
        };
        unsigned gt = 0;   // tip blocks consumed
        // per-pattern inputs of an op: tip state codes and exponents of the
        // children read from HBM, loaded one op ahead
        auto op_inputs = [&](const FuseOp& o, int p, int* sv, int* ev) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                sv[c] = o.kind[c] == kTipStates ? (int)a.tips[(size_t)o.child[c] * a.Ppad + p] : 0;
                ev[c] = (o.kind[c] == kInternal && o.prev != c)
                            ? a.epool[(size_t)o.child[c] * a.Ppad + p] : 0;
            }
        };
        for (int tile = blockIdx.x; ok && tile < a.n_tiles; tile += gridDim.x) {
            const int p = tile * kTcM + row;
            int cum_prev = 0;
            int sv_n[2] = {0, 0}, ev_n[2] = {0, 0};
            if (n_ops > 0) op_inputs(ops[0], p, sv_n, ev_n);
            for (int k = 0; ok && k < n_ops; ++k, ++nop) {
                const FuseOp o = ops[k];
                int cum = 0, sidx[2] = {sv_n[0], sv_n[1]};
                bool amb[2] = {false, false};
                for (int c = 0; c < 2; ++c) {
                    if (o.kind[c] == kInternal) cum += (o.prev == c) ? cum_prev : ev_n[c];
                    if (o.kind[c] == kTipStates) amb[c] = !(sidx[c] >= 0 && sidx[c] < a.S);
                }
                if (k + 1 < n_ops) op_inputs(ops[k + 1], p, sv_n, ev_n);
                // a tip's row of P^T (+ the lo row with split matrices) from the
                // block the TMA warp staged (128-byte swizzle: 16-byte unit j
                // of row s sits at unit j ^ (s & 7)), or the row sums of P for
                // an ambiguous code; false if the wait for the block gave up
                auto lookup64 = [&](int c, int r, float* v) -> bool {
                    const int ts = gt % 2;
                    const bool got = mbar_wait_or_abort(&tip_full[ts], (gt / 2) & 1, abort_v);
                    if (!__all_sync(0xffffffffu, got)) return false;
                    const unsigned char* tb = tip_area + ts * FusePipe<SPLIT>::tip_bytes;
                    if (amb[c]) {
                        const float* src =
                            a.rowsum + (size_t)(o.look[c] / ((SPLIT ? 4 : 2) * R * kTcN * kTcN)) *
                                           R * kTcN + (size_t)r * kTcN;
                        const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const float4 f = __ldg(s4 + u);
                            v[4 * u] = f.x;
                            v[4 * u + 1] = f.y;
                            v[4 * u + 2] = f.z;
                            v[4 * u + 3] = f.w;
                        }
                    } else {
                        const int sr = sidx[c];
#pragma unroll
                        for (int h = 0; h < 2; ++h)
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int off = h * kBChunk + sr * 128 + ((j ^ (sr & 7)) << 4);
                                float4 f = *reinterpret_cast<const float4*>(tb + off);
                                if (SPLIT) {
                                    const float4 l =
                                        *reinterpret_cast<const float4*>(tb + 2 * kBChunk + off);
                                    f.x += l.x;
                                    f.y += l.y;
                                    f.z += l.z;
                                    f.w += l.w;
                                }
                                const int i = h * 32 + j * 4;
                                v[i] = f.x;
                                v[i + 1] = f.y;
                                v[i + 2] = f.z;
                                v[i + 3] = f.w;
                            }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&tip_empty[ts]);
                    ++gt;
                    return true;
                };
                // pass 1: products of the two children per category, their
                // maximum; the unscaled products go to the A columns
                float m = 0.f;
                for (int r = 0; r < R; ++r, ++cat) {
                    const int b = cat & 1;
                    // every lane takes the same branch (the TMEM loads below
                    // are warp-collective), so a wait that gave up in any
                    // lane stops the whole warp
                    const bool got = mbar_wait_or_abort(&acc_full[b], (cat >> 1) & 1, abort_v);
                    if (!__all_sync(0xffffffffu, got)) {
                        ok = false;
                        if (lane == 0) atomicOr(&abort_sh, 8);
                        break;
                    }
                    tc_fence_after();
                    float x[64], y[64];
                    const uint32_t acc = lane_base + (uint32_t)(kPrevCols + b * 2 * kTcN);
                    bool got2 = true;
                    if (on_mma(o, 0)) tmem_ld64(acc, x);
                    else got2 = lookup64(0, r, x);
                    if (got2 && on_mma(o, 1)) tmem_ld64(acc + kTcN, y);
                    else if (got2) got2 = lookup64(1, r, y);
                    if (!got2) {
                        ok = false;
                        if (lane == 0) atomicOr(&abort_sh, 128);
                        break;
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[b]);
#pragma unroll
                    for (int i = 0; i < 64; ++i) {
                        x[i] *= y[i];
                        m = fmaxf(m, x[i]);
                    }
                    tmem_st64(lane_base + (uint32_t)(r * kTcN), x);
                }
                if (!ok) break;
                // pass 2: rescale, round to TF32, keep on chip and store
                float f1 = 1.f, f2 = 1.f;
                if (a.rescale) cum += post_scale(m, &f1, &f2);
                // row 0 of this warp's 32 patterns in the output buffer
                float* dst = a.pool + (size_t)o.dest * a.bstride +
                             (size_t)(tile * kTcM + quarter * 32) * kTcN;
                for (int r = 0; r < R; ++r) {
                    float z[64];
                    tmem_ld64(lane_base + (uint32_t)(r * kTcN), z);
#pragma unroll
                    for (int i = 0; i < 64; ++i) z[i] = to_tf32(z[i] * f1 * f2);
                    tmem_st64(lane_base + (uint32_t)(r * kTcN), z);
                    store_row(dst + (size_t)r * a.Ppad * kTcN, z);
                }
                a.epool[(size_t)o.dest * a.Ppad + p] = cum;
                cum_prev = cum;
                // this warp's rows of the op are done and may be read from
                // TMEM, and its stores by the copy engine (each warp
                // publishes its own count: no barrier among the epilogue
                // warps, which an abort could leave unmatched)
                fence_proxy_async_global();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) st_release_cta(&ready_sh[quarter], nop + 1);
            }
        }
        if (warp == 2 && lane == 0) tip_used_sh = gt;
    }
    __syncthreads();
    if (abort_sh && tid == 0) {
        atomicOr(a.err, (abort_sh & 0xff) | (1 << 11));
        // bounded drain of copies still in flight
        for (unsigned g = used_sh; g < loads_sh; ++g) mbar_wait(&full[g % kSt], (g / kSt) & 1);
        for (unsigned g = tip_used_sh; g < tip_loads_sh; ++g) mbar_wait(&tip_full[g % 2], (g / 2) & 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
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
    const size_t mrows =
        ((size_t)I->n_mats * blocks_per_slot(I) + (size_t)I->n_models * blocks_per_q(I)) * I->R * kTcN;
    if ((rc = make_map(I, &m[2], I->d_matw, mrows, kTcN))) return rc;
    m[1] = m[0];  // tip-partials map until a tip pool exists
    return TL_OK;
}

size_t tc_matw_floats(const Instance* I) {
    return (size_t)I->n_mats * I->matw_stride +
           (size_t)I->n_models * blocks_per_q(I) * I->R * kTcN * kTcN;
}

int tc_set_tip_pool(Instance* I) {
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(I->tmaps.data());
    return make_map(I, &m[1], I->tc_tip_pool, (size_t)I->n_tips * I->R * I->Ppad, kTcM);
}

int launch_q_tc(Instance* I, int model) {
    float* dst = reinterpret_cast<float*>(I->d_matw) + (size_t)qrow_of(I, model) * kTcN;
    k_q_tc<<<1, 256, 0, I->stream>>>(I->models[model].Q, dst, I->R, I->split);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "tensor-core Q copy");
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
            tc_operand(I, t, 0, ops[k].child1, ops[k].mat1);
            tc_operand(I, t, 1, ops[k].child2, ops[k].mat2);
            t.dest = ops[k].dest - I->n_tips;
            t.qin = -1;
            t.uout[0] = t.uout[1] = t.edge[0] = t.edge[1] = -1;
            dev.push_back(t);
        }
    }
    first[n_levels] = (int)dev.size();
    if (dev.size() * sizeof(TcOp) > cap) return fail(I, TL_ERR_ARG, "op area too small");
    int rc = upload_bytes(I, d_ops_area, dev.data(), dev.size() * sizeof(TcOp));
    if (rc) return rc;
    TcArgs a = tc_args(I);
    const TcOp* d = reinterpret_cast<const TcOp*>(d_ops_area);
    for (int L = 0; L < n_levels; ++L) launch_mode<kPost>(I, d + first[L], first[L + 1] - first[L], a);
    return cuda_check(I, cudaGetLastError(), "tensor-core post-order kernel");
}

// The subtree-fused post-order kernel is used for TF32 instances with TF32
// storage (plain or split matrices) unless TL_TC_FUSED=0; split partials
// need an A_lo tile per operand, which has no room in tensor memory beside
// the on-chip result, and take the level-by-level kernels.
int tc_fused_enabled(const Instance* I) {
    const char* e = getenv("TL_TC_FUSED");   // read per call: tests compare both kernels
    return (!e || atoi(e) != 0) && I->prec == kTF32 && !I->split_partials;
}

int launch_post_tc_fused(Instance* I, const DevPostOp* plan_ops, int n, void* d_ops_area,
                         size_t cap) {
    std::vector<FuseOp> dev(n);
    std::vector<int> writer(I->n_buffers, -1);   // op of this list storing each buffer
    for (int k = 0; k < n; ++k) writer[plan_ops[k].dest] = k;
    for (int k = 0; k < n; ++k) {
        const DevPostOp& d = plan_ops[k];
        FuseOp& f = dev[k];
        std::memset(&f, 0, sizeof f);
        f.prev = -1;
        for (int c = 0; c < 2; ++c) {
            f.child[c] = d.child[c];
            f.kind[c] = d.kind[c];
            f.brow[c] = brow_of(I, d.mat[c], 0);
            f.look[c] = look_of(I, d.mat[c], 1);
            f.tbrow[c] = brow_of(I, d.mat[c], 1);
            f.src[c] = -1;
            if (d.kind[c] == kInternal) {
                if (d.slot_in[c] == kFromRegisters) f.prev = c;
                else f.src[c] = writer[d.child[c]] < k ? writer[d.child[c]] : -1;
            }
        }
        f.dest = d.dest;
    }
    if (dev.size() * sizeof(FuseOp) > cap) return fail(I, TL_ERR_ARG, "op area too small");
    int rc = upload_bytes(I, d_ops_area, dev.data(), dev.size() * sizeof(FuseOp));
    if (rc) return rc;
    TcArgs a = tc_args(I);
    int sms = 0, dev_id = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    const int grid = std::max(1, std::min(a.n_tiles, sms));
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(I->tmaps.data());
    const FuseOp* d = reinterpret_cast<const FuseOp*>(d_ops_area);
    if (I->split) {
        const size_t smem = FusePipe<true>::smem + 1024;
        cudaFuncSetAttribute(k_tc_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tc_fused<true><<<grid, kFuseThreads, smem, I->stream>>>(m[0], m[1], m[2], d, n, a);
    } else {
        const size_t smem = FusePipe<false>::smem + 1024;
        cudaFuncSetAttribute(k_tc_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tc_fused<false><<<grid, kFuseThreads, smem, I->stream>>>(m[0], m[1], m[2], d, n, a);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "fused tensor-core post-order kernel");
}

// Pre-order pass with gradient, level by level from the root: PRE1 per
// parent (v = P x, den, u = q o v_sibling, tip gradients), then PRE2 per
// internal child (q = u P, Q x, internal gradients, q rescaled in place).
int launch_pre_tc(Instance* I, const tl_pre_op* ops, int n, const int* edge_row, int model,
                  double* d_gpart, void* d_ops_area, size_t cap, int dgen) {
    std::vector<int> prod(I->n_bufs, -1), level(n, 0);
    for (int k = 0; k < n; ++k) {
        if (ops[k].parent_pre >= 0 && prod[ops[k].parent_pre] >= 0)
            level[k] = level[prod[ops[k].parent_pre]] + 1;
        for (int c = 0; c < 2; ++c)
            if (ops[k].pre[c] >= 0) prod[ops[k].pre[c]] = k;
    }
    const int n_levels = n ? *std::max_element(level.begin(), level.end()) + 1 : 0;
    std::vector<TcOp> dev;
    std::vector<int> f1(n_levels), n1(n_levels), f2(n_levels), n2(n_levels);
    for (int L = 0; L < n_levels; ++L) {
        f1[L] = (int)dev.size();
        std::vector<TcOp> second;
        for (int k = 0; k < n; ++k) {
            if (level[k] != L) continue;
            const tl_pre_op& o = ops[k];
            TcOp t;
            std::memset(&t, 0, sizeof t);
            for (int c = 0; c < 2; ++c) {
                tc_operand(I, t, c, o.child[c], o.mat[c]);
                if (t.kind[c] == kTipPartials)
                    return fail(I, TL_ERR_UNSUPPORTED,
                                "TL_PREC_TF32 pre-order pass: tips must hold states");
                t.uout[c] = -1;
                t.edge[c] = -1;
                if (t.kind[c] == kTipStates) {
                    t.edge[c] = o.edge[c] >= 0 ? edge_row[o.edge[c]] : -1;
                    t.dlook[c] = o.dmat[c] >= 0 ? look_of(I, o.dmat[c], 1) : 0;
                    if (t.edge[c] >= 0 && o.dmat[c] < 0)
                        return fail(I, TL_ERR_ARG, "pre op %d: edge without dmat", k);
                } else {
                    if (o.pre[c] < 0)
                        return fail(I, TL_ERR_ARG, "TL_PREC_TF32: internal child of pre op %d needs "
                                    "a pre buffer", k);
                    t.uout[c] = o.pre[c] - I->n_tips;
                    TcOp u;
                    std::memset(&u, 0, sizeof u);
                    u.kind[0] = kInternal;
                    u.child[0] = t.uout[c];
                    u.brow[0] = brow_of(I, o.mat[c], 1);       // q = u P  (B = P^T)
                    u.kind[1] = kInternal;
                    u.child[1] = o.child[c] - I->n_tips;       // Q x_c, or dP x_c
                    u.brow[1] = dgen ? brow_of(I, o.dmat[c], 0) : qrow_of(I, model);
                    if (dgen && o.dmat[c] < 0 && o.edge[c] >= 0)
                        return fail(I, TL_ERR_ARG, "pre op %d: edge without dmat", k);
                    if (dgen && o.dmat[c] < 0) u.brow[1] = qrow_of(I, model);
                    u.dest = t.uout[c];
                    u.qin = -1;
                    u.uout[0] = u.uout[1] = -1;
                    u.edge[0] = o.edge[c] >= 0 ? edge_row[o.edge[c]] : -1;
                    u.edge[1] = -1;
                    second.push_back(u);
                }
            }
            t.qin = o.parent_pre >= 0 ? o.parent_pre - I->n_tips : -1;
            t.dest = 0;
            dev.push_back(t);
        }
        n1[L] = (int)dev.size() - f1[L];
        f2[L] = (int)dev.size();
        dev.insert(dev.end(), second.begin(), second.end());
        n2[L] = (int)dev.size() - f2[L];
    }
    if (dev.size() * sizeof(TcOp) > cap) return fail(I, TL_ERR_ARG, "op area too small");
    int rc = upload_bytes(I, d_ops_area, dev.data(), dev.size() * sizeof(TcOp));
    if (rc) return rc;
    TcArgs a = tc_args(I);
    a.pi = I->models[model].pi;
    a.gpart = d_gpart;
    a.dgen = dgen;
    const TcOp* d = reinterpret_cast<const TcOp*>(d_ops_area);
    for (int L = 0; L < n_levels; ++L) {
        if (n1[L]) launch_mode<kPre1>(I, d + f1[L], n1[L], a);
        if (n2[L]) launch_mode<kPre2>(I, d + f2[L], n2[L], a);
    }
    return cuda_check(I, cudaGetLastError(), "tensor-core pre-order kernels");
}

int launch_root_tc(Instance* I, int root_pool, int model, double* d_site, double* d_part,
                   int n_parts) {
    TcArgs a = tc_args(I);
    const float* x = a.pool + (size_t)root_pool * a.bstride;
    const int* ep = a.epool + (size_t)root_pool * a.Ppad;
    double* catw = I->d_tmp;  // staged by the caller
    k_root_tc<<<n_parts, 128, 0, I->stream>>>(x, ep, I->models[model].pi, a, I->d_patw, I->P,
                                              d_site, d_part, catw, I->d_err + 1);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "tensor-core root kernel");
}

}  // namespace tl
