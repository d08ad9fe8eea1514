// Four-state (nucleotide) kernels: post-order pruning with per-pattern
// power-of-two rescaling, root log-likelihood, fused pre-order pass with
// branch-length gradient, and edge derivatives from stored partials.
//
// Design: patterns are independent given the tree (Sec. "Benchmarks on
// NVIDIA and AMD GPUs": the alignment splits into conditionally independent
// blocks), so a warp owns a tile of patterns and walks the WHOLE operation
// list for it in a single launch; no warp ever waits for another. LPP lanes
// share a pattern, one rate category each (LPP = 4 for four categories: a
// warp tile is 8 patterns), so per-pattern maxima and sums over categories
// are LPP-lane shuffles. The grid is persistent (sized by occupancy) and
// warps stride over tiles. A child produced by the op just before is taken
// from registers, one produced earlier in the same list from a warp-private
// shared-memory slot (the host assigns both); only results the caller asked
// for go to HBM. Partials are [category][pattern][4] so a warp's float4 /
// double2x2 accesses cover LPP runs of consecutive patterns. A tip with
// states uses a column of P (or the row sums for an ambiguous code) instead
// of a product.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "tl_internal.cuh"

namespace tl {

template <typename T>
struct V4 {
    T x, y, z, w;
};

__device__ __forceinline__ V4<float> ld4(const float* p) {
    float4 v = *reinterpret_cast<const float4*>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
    double2 a = *reinterpret_cast<const double2*>(p);
    double2 b = *reinterpret_cast<const double2*>(p + 2);
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ V4<float> ldg4(const float* p) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ldg4(const double* p) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(float* p, V4<float> v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ void st4(double* p, V4<double> v) {
    *reinterpret_cast<double2*>(p) = make_double2(v.x, v.y);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v.z, v.w);
}

template <typename T>
__device__ __forceinline__ V4<T> mul(V4<T> a, V4<T> b) {
    return {a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w};
}
template <typename T>
__device__ __forceinline__ T dot(V4<T> a, V4<T> b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
template <typename T>
__device__ __forceinline__ T vmax(V4<T> a) {
    return fmax(fmax(a.x, a.y), fmax(a.z, a.w));
}
// max(a, b, c) in one instruction for FP32 (sm_100 and later)
__device__ __forceinline__ float max3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ double max3(double a, double b, double c) { return fmax(fmax(a, b), c); }
// the largest of the CPL V4 values (a tree of three-input maxima)
template <int CPL, typename T>
__device__ __forceinline__ T vmax_all(const V4<T>* v) {
    if constexpr (CPL == 4) {
        const T a = max3(v[0].x, v[0].y, v[0].z), b = max3(v[0].w, v[1].x, v[1].y);
        const T c = max3(v[1].z, v[1].w, v[2].x), d = max3(v[2].y, v[2].z, v[2].w);
        const T e = max3(v[3].x, v[3].y, v[3].z);
        return max3(max3(a, b, c), max3(d, e, v[3].w), T(0));
    } else {
        T m = vmax(v[0]);
#pragma unroll
        for (int j = 1; j < CPL; ++j) m = fmax(m, vmax(v[j]));
        return m;
    }
}

// ---- packed FP32 pairs (fma/mul/add .f32x2 of sm_100 and later): two
// lanes of a V4<float> per instruction, each rounded exactly as the scalar
// instruction would, so a packed chain gives the scalar chain's bits.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ V4<float> mul(V4<float> a, V4<float> b) {
    V4<float> r;
    upk2(mul2(pk2(a.x, a.y), pk2(b.x, b.y)), r.x, r.y);
    upk2(mul2(pk2(a.z, a.w), pk2(b.z, b.w)), r.z, r.w);
    return r;
}
// (a.x b.x + a.z b.z) + (a.y b.y + a.w b.w)
__device__ __forceinline__ float dot(V4<float> a, V4<float> b) {
    float lo, hi;
    upk2(fma2(pk2(a.z, a.w), pk2(b.z, b.w), mul2(pk2(a.x, a.y), pk2(b.x, b.y))), lo, hi);
    return lo + hi;
}

// P x with P given by its columns c0..c3 (column j at col + j * cs):
// x0 c0 + x1 c1 + x2 c2 + x3 c3.
template <typename T>
__device__ __forceinline__ V4<T> matvec(const T* col, int cs, V4<T> x) {
    V4<T> c0 = ld4(col), c1 = ld4(col + cs), c2 = ld4(col + 2 * cs), c3 = ld4(col + 3 * cs);
    V4<T> r;
    r.x = x.x * c0.x + x.y * c1.x + x.z * c2.x + x.w * c3.x;
    r.y = x.x * c0.y + x.y * c1.y + x.z * c2.y + x.w * c3.y;
    r.z = x.x * c0.z + x.y * c1.z + x.z * c2.z + x.w * c3.z;
    r.w = x.x * c0.w + x.y * c1.w + x.z * c2.w + x.w * c3.w;
    return r;
}
// P^T u: component j is column j . u
template <typename T>
__device__ __forceinline__ V4<T> matTvec(const T* col, int cs, V4<T> u) {
    V4<T> c0 = ld4(col), c1 = ld4(col + cs), c2 = ld4(col + 2 * cs), c3 = ld4(col + 3 * cs);
    return {dot(c0, u), dot(c1, u), dot(c2, u), dot(c3, u)};
}
template <typename T>
__device__ __forceinline__ V4<T> matvec_cols(V4<T> c0, V4<T> c1, V4<T> c2, V4<T> c3, V4<T> x) {
    V4<T> r;
    r.x = x.x * c0.x + x.y * c1.x + x.z * c2.x + x.w * c3.x;
    r.y = x.x * c0.y + x.y * c1.y + x.z * c2.y + x.w * c3.y;
    r.z = x.x * c0.z + x.y * c1.z + x.z * c2.z + x.w * c3.z;
    r.w = x.x * c0.w + x.y * c1.w + x.z * c2.w + x.w * c3.w;
    return r;
}
// The FP32 matvec as packed pairs, in the scalar chain's order (same bits).
__device__ __forceinline__ V4<float> matvec_cols(V4<float> c0, V4<float> c1, V4<float> c2,
                                                 V4<float> c3, V4<float> x) {
    const f32x2 sx = pk2(x.x, x.x), sy = pk2(x.y, x.y), sz = pk2(x.z, x.z), sw = pk2(x.w, x.w);
    f32x2 a = mul2(sx, pk2(c0.x, c0.y)), b = mul2(sx, pk2(c0.z, c0.w));
    a = fma2(sy, pk2(c1.x, c1.y), a);
    b = fma2(sy, pk2(c1.z, c1.w), b);
    a = fma2(sz, pk2(c2.x, c2.y), a);
    b = fma2(sz, pk2(c2.z, c2.w), b);
    a = fma2(sw, pk2(c3.x, c3.y), a);
    b = fma2(sw, pk2(c3.z, c3.w), b);
    V4<float> r;
    upk2(a, r.x, r.y);
    upk2(b, r.z, r.w);
    return r;
}
__device__ __forceinline__ V4<float> matvec(const float* col, int cs, V4<float> x) {
    return matvec_cols(ld4(col), ld4(col + cs), ld4(col + 2 * cs), ld4(col + 3 * cs), x);
}

// frexp exponent e of m >= 0 (m = f 2^e, f in [0.5, 1)); 0 for m == 0.
__device__ __forceinline__ int frexp_exp(float m) {
    int E = (__float_as_int(m) >> 23) & 0xff;
    if (E == 0) {
        if (m == 0.f) return 0;
        E = ((__float_as_int(m * 18446744073709551616.f) >> 23) & 0xff) - 64;
    }
    return E - 126;
}
__device__ __forceinline__ int frexp_exp(double m) {
    int E = (int)((__double_as_longlong(m) >> 52) & 0x7ff);
    if (E == 0) {
        if (m == 0.0) return 0;
        E = (int)((__double_as_longlong(m * 18446744073709551616.0) >> 52) & 0x7ff) - 64;
    }
    return E - 1022;
}
// exact multiplication by 2^k (two steps when 2^k is not a normal number)
__device__ __forceinline__ float pow2(float, int k) { return __int_as_float((k + 127) << 23); }
__device__ __forceinline__ double pow2(double, int k) {
    return __longlong_as_double((long long)(k + 1023) << 52);
}
template <typename T>
__device__ __forceinline__ void scale_by_pow2(V4<T>* v, int n, int k) {
    const int lim = sizeof(T) == 4 ? 126 : 1022;
    if (k >= -lim && k <= lim) {
        T f = pow2(T(0), k);
        for (int r = 0; r < n; ++r) v[r] = {v[r].x * f, v[r].y * f, v[r].z * f, v[r].w * f};
    } else {
        int k1 = k / 2;
        T f1 = pow2(T(0), k1), f2 = pow2(T(0), k - k1);
        for (int r = 0; r < n; ++r)
            v[r] = {v[r].x * f1 * f2, v[r].y * f1 * f2, v[r].z * f1 * f2, v[r].w * f1 * f2};
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// a / b for the gradient ratios: FP32 by the fast division (at most 2 ulp,
// b well inside the normal range here), FP64 exactly
__device__ __forceinline__ float ratio_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double ratio_div(double a, double b) { return a / b; }
__device__ __forceinline__ int tip_col(int8_t s) { return (s >= 0 && s < 4) ? (int)s : 4; }

// ---------------------------------------------------------------------------
// batched launches: one launch walks the op lists of several instances.
// Warps claim global tiles from a counter (largest jobs first, so the long
// walks start in the first wave), find the owning job by binary search and
// stage its arguments in a warp-private shared-memory copy. A job's tiles
// are computed exactly as in its own launch, so results do not depend on
// what else is in the batch.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ bool batch_claim(const BatchRef<T>& br, int total, BatchJob<T>* stage,
                                            int& cur, int& tile, int lane) {
    int g = 0;
    if (lane == 0) g = atomicAdd(br.counter, 1);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= total) return false;
    int lo = 0, hi = br.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(br.tile_begin + mid) <= g) lo = mid;
        else hi = mid - 1;
    }
    if (lo != cur) {
        __syncwarp();  // every lane is done with the previous job's copy
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(br.jobs + lo);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(stage);
        for (int i = lane; i < (int)(sizeof(BatchJob<T>) / 8); i += 32) dst[i] = __ldg(src + i);
        __syncwarp();
        cur = lo;
    }
    tile = g - __ldg(br.tile_begin + lo);
    return true;
}

// The arguments a tile is computed with: the kernel parameter, or the
// staged job.
template <bool BATCH, typename T>
__device__ __forceinline__ const NucArgs<T>& pick_args(const NucArgs<T>& param,
                                                       const BatchJob<T>* stage) {
    if constexpr (BATCH) return stage->a;
    else return param;
}

// ---------------------------------------------------------------------------
// post-order
// ---------------------------------------------------------------------------
// Loads that feed op k (tip states, partials read from memory) are issued
// while op k - 1 computes. Without this every op waits a full DRAM round
// trip for its inputs.

// Children and their kinds: the first 16 bytes of a post- or pre-order op.
template <typename Op>
__device__ __forceinline__ int4 op_head(const Op* ops, int k, int n) {
    return (k < n) ? __ldg(reinterpret_cast<const int4*>(ops + k)) : make_int4(0, 0, -1, -1);
}
template <typename T>
__device__ __forceinline__ int tip_state(const NucArgs<T>& a, int child, int kind, int p) {
    return kind == kTipStates ? (int)__ldg(a.tips + (size_t)child * a.Ppad + p) : 0;
}

// ---------------------------------------------------------------------------
// per-warp copy pipeline: op descriptors two ops ahead and the matrices of
// the next op are copied into warp-private shared memory with cp.async while
// the current op computes; completion is the hardware wait_group (no spin).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ V4<T> lds4(const T* p) {
    return ld4(p);
}

// NMAT matrices per op (post: P of both children; pre: P and dP of both),
// each `matf` elements (all categories); obuf holds three descriptors.
template <typename Op, typename T, int NMAT>
struct WarpPipe {
    Op* obuf;
    T* mbuf;
    int matf;
    int per;       // 16-byte chunks per matrix
    int m0, c0;    // this lane's first chunk: matrix m0, chunk c0 (lane = m0 per + c0)
    __device__ __forceinline__ void init(int lane) {
        per = matf * (int)sizeof(T) / 16;
        m0 = lane / per;
        c0 = lane - m0 * per;
    }
    __device__ __forceinline__ void issue_op(const Op* ops, int j, int n, int lane) {
        constexpr int chunks = sizeof(Op) / 16;
        if (j < n && lane < chunks)
            cp_async16(reinterpret_cast<char*>(obuf + j % 3) + lane * 16,
                       reinterpret_cast<const char*>(ops + j) + lane * 16);
    }
    // idx: the NMAT matrix slots (-1: none). A lane's chunks are lane,
    // lane + 32, ...; the slot is picked by selects, not by indexing, so idx
    // stays in registers when it is a local array.
    __device__ __forceinline__ void issue_mats(int j, int n, const int* idx, const T* mat,
                                               int mat_stride, int lane) {
        if (j >= n) return;
        T* dst = mbuf + (j & 1) * NMAT * matf;
        int slots[NMAT];
#pragma unroll
        for (int m = 0; m < NMAT; ++m) slots[m] = idx[m];
        // the lane's chunks lane, lane + 32, ... walked as (matrix, chunk)
        // pairs: no division per chunk
        int m = m0, c = c0;
        while (m < NMAT) {
            int slot = slots[0];
#pragma unroll
            for (int i = 1; i < NMAT; ++i)
                if (m == i) slot = slots[i];
            if (slot >= 0)
                cp_async16(reinterpret_cast<char*>(dst + m * matf) + c * 16,
                           reinterpret_cast<const char*>(mat + (size_t)slot * mat_stride) + c * 16);
            c += 32;
            while (c >= per) {
                c -= per;
                ++m;
            }
        }
        (void)lane;
    }
    __device__ __forceinline__ const T* mats(int k) const { return mbuf + (k & 1) * NMAT * matf; }
};

template <typename Op, typename T, int NMAT>
__host__ __device__ constexpr size_t pipe_bytes(int R) {
    return 3 * sizeof(Op) + 2 * (size_t)NMAT * kColStride * 4 * R * sizeof(T);
}

// Lane layout of the post- and pre-order kernels: LPP lanes share a
// pattern and each holds CPL categories (r = r0 + j * LPP, j < CPL), so a
// warp tile has 32 / LPP patterns. Fewer lanes per pattern amortise the
// per-op work (op fetch, addressing, control) over more patterns; more lanes
// lower the registers each lane needs.
// BATCH: `a_` gives the shared-memory layout (the largest slot count of the
// jobs, their common R) and the total tile count; each tile's arguments and
// ops come from its job in `br`.
// PPL: patterns per lane. A warp tile is PPL sub-tiles of 32 / LPP
// consecutive patterns; a lane computes the same categories of one pattern
// in each, so the per-op work that does not depend on the pattern (op and
// matrix fetches, matrix columns from shared memory, control) is shared by
// PPL patterns.
template <typename T, int LPP, int CPL, int NR, bool BATCH, int PPL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_post4(const DevPostOp* __restrict__ ops_, int n_ops_, const __grid_constant__ NucArgs<T> a_,
        const BatchRef<T> br) {
    constexpr int TP = 32 / LPP;
    // NR > 0: the category count is a compile-time constant
    constexpr bool kFull = NR > 0 && LPP * CPL == NR;
    constexpr int SL = PPL * CPL;  // V4 values per lane in one slot
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = lane % LPP, pp = lane / LPP;
    const int R = NR > 0 ? NR : a_.R;
    const int cs = R * 4;  // matrix column stride (all categories of a column)
    bool act[CPL];
#pragma unroll
    for (int j = 0; j < CPL; ++j) act[j] = kFull || (r0 + j * LPP < R);
    V4<T>* slots = reinterpret_cast<V4<T>*>(smem_raw) + (size_t)warp * a_.n_slots * SL * 32;
    int* sexp = reinterpret_cast<int*>(reinterpret_cast<V4<T>*>(smem_raw) +
                                       (size_t)kWarpsPerBlock * a_.n_slots * SL * 32) +
                warp * a_.n_slots * PPL * 32;
    unsigned char* pipe_base = reinterpret_cast<unsigned char*>(
        reinterpret_cast<int*>(reinterpret_cast<V4<T>*>(smem_raw) +
                               (size_t)kWarpsPerBlock * a_.n_slots * SL * 32) +
        kWarpsPerBlock * a_.n_slots * PPL * 32);
    WarpPipe<DevPostOp, T, 2> pipe;
    pipe.obuf = reinterpret_cast<DevPostOp*>(pipe_base + (size_t)warp * pipe_bytes<DevPostOp, T, 2>(R));
    pipe.mbuf = reinterpret_cast<T*>(pipe.obuf + 3);
    pipe.matf = kColStride * 4 * R;
    pipe.init(lane);
    BatchJob<T>* stage = reinterpret_cast<BatchJob<T>*>(
        pipe_base + (size_t)kWarpsPerBlock * pipe_bytes<DevPostOp, T, 2>(R)) + warp;
    const NucArgs<T>& a = pick_args<BATCH>(a_, stage);
    const V4<T> zero = {T(0), T(0), T(0), T(0)};
    const int nw = gridDim.x * kWarpsPerBlock;
    const DevPostOp* ops = ops_;
    int n_ops = n_ops_;
    int cur = -1;
    for (int next = blockIdx.x * kWarpsPerBlock + warp; BATCH || next < a_.n_tiles; next += nw) {
        int tile = next;
        if constexpr (BATCH) {
            if (!batch_claim(br, a_.n_tiles, stage, cur, tile, lane)) break;
            ops = static_cast<const DevPostOp*>(stage->ops);
            n_ops = stage->n_ops;
        }
        int p[PPL];
        size_t off0[PPL];
#pragma unroll
        for (int i = 0; i < PPL; ++i) {
            p[i] = (tile * PPL + i) * TP + pp;
            off0[i] = ((size_t)r0 * a.Ppad + p[i]) * 4;  // category r0
        }
        const size_t offj = (size_t)LPP * a.Ppad * 4;    // next category of this lane
        V4<T> prev[PPL][CPL];
        int prev_cum[PPL];
#pragma unroll
        for (int i = 0; i < PPL; ++i) {
            prev_cum[i] = 0;
#pragma unroll
            for (int j = 0; j < CPL; ++j) prev[i][j] = zero;
        }
        // tip states of the current op (A) and the next one (B)
        int tsA[2][PPL], tsB[2][PPL];
        {
            const int4 h = op_head(ops, 0, n_ops);
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                tsA[0][i] = tip_state(a, h.x, h.z, p[i]);
                tsA[1][i] = tip_state(a, h.y, h.w, p[i]);
            }
        }
        // pipeline prologue: descriptors 0 and 1, then matrices of op 0
        __syncwarp();
        pipe.issue_op(ops, 0, n_ops, lane);
        pipe.issue_op(ops, 1, n_ops, lane);
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        pipe.issue_mats(0, n_ops, pipe.obuf[0].mat, a.mat, a.mat_stride, lane);
        cp_async_commit();
        auto op_body = [&](int k, int (&ts)[2][PPL], int (&tn)[2][PPL]) {
            cp_async_wait_all();
            __syncwarp();
            pipe.issue_op(ops, k + 2, n_ops, lane);
            if (k + 1 < n_ops)
                pipe.issue_mats(k + 1, n_ops, pipe.obuf[(k + 1) % 3].mat, a.mat, a.mat_stride, lane);
            cp_async_commit();
            {
                const int4 hn = op_head(ops, k + 1, n_ops);
#pragma unroll
                for (int i = 0; i < PPL; ++i) {
                    tn[0][i] = tip_state(a, hn.x, hn.z, p[i]);
                    tn[1][i] = tip_state(a, hn.y, hn.w, p[i]);
                }
            }
            const DevPostOp op = pipe.obuf[k % 3];
            const T* mk = pipe.mats(k);
            V4<T> acc[PPL][CPL];
            int cum[PPL];
#pragma unroll
            for (int i = 0; i < PPL; ++i) cum[i] = 0;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const T* mc = mk + c * pipe.matf + r0 * 4;
                V4<T> v[PPL][CPL];
                if (op.kind[c] == kTipStates) {
#pragma unroll
                    for (int i = 0; i < PPL; ++i) {
                        const int col = tip_col((int8_t)ts[c][i]);
#pragma unroll
                        for (int j = 0; j < CPL; ++j)
                            v[i][j] = act[j] ? lds4(mc + col * cs + j * LPP * 4) : zero;
                    }
                } else {
                    V4<T> x[PPL][CPL];
                    const int si = op.slot_in[c];
                    if (si == kFromRegisters) {
#pragma unroll
                        for (int i = 0; i < PPL; ++i) {
#pragma unroll
                            for (int j = 0; j < CPL; ++j) x[i][j] = prev[i][j];
                            cum[i] += prev_cum[i];
                        }
                    } else if (si >= 0) {
#pragma unroll
                        for (int i = 0; i < PPL; ++i) {
#pragma unroll
                            for (int j = 0; j < CPL; ++j)
                                x[i][j] = slots[((si * PPL + i) * CPL + j) * 32 + lane];
                            cum[i] += sexp[(si * PPL + i) * 32 + lane];
                        }
                    } else {
                        const T* b = (op.kind[c] == kTipPartials)
                                         ? a.tipbuf[op.child[c]]
                                         : a.pool + (size_t)op.child[c] * a.bstride;
#pragma unroll
                        for (int i = 0; i < PPL; ++i) {
#pragma unroll
                            for (int j = 0; j < CPL; ++j)
                                x[i][j] = act[j] ? ld4(b + off0[i] + j * offj) : zero;
                            if (op.kind[c] == kInternal)
                                cum[i] += a.epool[(size_t)op.child[c] * a.Ppad + p[i]];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < CPL; ++j) {
                        if (act[j]) {
                            // the columns once for all PPL patterns
                            const T* col = mc + j * LPP * 4;
                            const V4<T> c0 = lds4(col), c1 = lds4(col + cs), c2 = lds4(col + 2 * cs),
                                        c3 = lds4(col + 3 * cs);
#pragma unroll
                            for (int i = 0; i < PPL; ++i) v[i][j] = matvec_cols(c0, c1, c2, c3, x[i][j]);
                        } else {
#pragma unroll
                            for (int i = 0; i < PPL; ++i) v[i][j] = zero;
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < PPL; ++i)
#pragma unroll
                    for (int j = 0; j < CPL; ++j) acc[i][j] = (c == 0) ? v[i][j] : mul(acc[i][j], v[i][j]);
            }
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                if (a.rescale) {
                    T m = vmax_all<CPL>(acc[i]);
#pragma unroll
                    for (int o = 1; o < LPP; o <<= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
                    const int e = frexp_exp(m);
                    if (e != 0) {
                        scale_by_pow2(acc[i], CPL, -e);
                        cum[i] += e;
                    }
                }
                if (op.store) {
                    T* d = a.pool + (size_t)op.dest * a.bstride + off0[i];
#pragma unroll
                    for (int j = 0; j < CPL; ++j)
                        if (act[j]) st4(d + j * offj, acc[i][j]);
                    if (r0 == 0) a.epool[(size_t)op.dest * a.Ppad + p[i]] = cum[i];
                }
                if (op.slot_out >= 0) {
#pragma unroll
                    for (int j = 0; j < CPL; ++j)
                        slots[((op.slot_out * PPL + i) * CPL + j) * 32 + lane] = acc[i][j];
                    sexp[(op.slot_out * PPL + i) * 32 + lane] = cum[i];
                }
#pragma unroll
                for (int j = 0; j < CPL; ++j) prev[i][j] = acc[i][j];
                prev_cum[i] = cum[i];
            }
        };
        for (int k = 0; k < n_ops; ++k) {
            op_body(k, tsA, tsB);
#pragma unroll
            for (int i = 0; i < PPL; ++i) {
                tsA[0][i] = tsB[0][i];
                tsA[1][i] = tsB[1][i];
            }
        }
        cp_async_wait_all();
    }
}

// Sum over the LPP lanes of one pattern (every lane of the group gets it).
template <int LPP, typename X>
__device__ __forceinline__ X group_sum(X v) {
#pragma unroll
    for (int o = 1; o < LPP; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Sum over the patterns of a warp tile of a value that is equal on the LPP
// lanes of each pattern.
template <int LPP, typename X = double>
__device__ __forceinline__ X tile_sum(X v) {
#pragma unroll
    for (int o = LPP; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// root log-likelihood: per-tile partial sums of w_p l_p
// ---------------------------------------------------------------------------
template <typename T, int LPP, bool BATCH>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_root4(int kind_, int root_, const __grid_constant__ NucArgs<T> a_, const double* __restrict__ pi_,
        double* __restrict__ site_, double* __restrict__ part_, int* __restrict__ err_,
        const BatchRef<T> br) {
    constexpr int TP = 32 / LPP;
    __shared__ BatchJob<T> stages[BATCH ? kWarpsPerBlock : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane % LPP, pp = lane / LPP;
    BatchJob<T>* stage = stages + (BATCH ? warp : 0);
    const NucArgs<T>& a = pick_args<BATCH>(a_, stage);
    const bool ract = r < a_.R;
    const int nw = gridDim.x * kWarpsPerBlock;
    int kind = kind_, root = root_;
    const double* pi = pi_;
    double *site = site_, *part = part_;
    int* err = err_;
    int cur = -1;
    for (int next = blockIdx.x * kWarpsPerBlock + warp; BATCH || next < a_.n_tiles; next += nw) {
        int tile = next;
        if constexpr (BATCH) {
            if (!batch_claim(br, a_.n_tiles, stage, cur, tile, lane)) break;
            kind = stage->root_kind;
            root = stage->root;
            pi = stage->pi;
            site = nullptr;
            part = stage->part;
            err = stage->err;
        }
        const int p = tile * TP + pp;
        double Lr = 0.0;
        int cum = 0;
        if (kind == kTipStates) {
            const int s = a.tips[(size_t)root * a.Ppad + p];
            double v = (s >= 0 && s < 4) ? pi[s] : pi[0] + pi[1] + pi[2] + pi[3];
            if (ract) Lr = (double)a.catw[r] * v;
        } else {
            if (ract) {
                const T* b = (kind == kTipPartials) ? a.tipbuf[root]
                                                    : a.pool + (size_t)root * a.bstride;
                V4<T> x = ld4(b + ((size_t)r * a.Ppad + p) * 4);
                Lr = (double)a.catw[r] * (pi[0] * (double)x.x + pi[1] * (double)x.y +
                                          pi[2] * (double)x.z + pi[3] * (double)x.w);
            }
            if (kind == kInternal) cum = a.epool[(size_t)root * a.Ppad + p];
        }
        const double L = group_sum<LPP>(Lr);
        const double l = log(L) + 0.69314718055994530942 * (double)cum;
        double contrib = 0.0;
        if (p < a.P) {
            if (r == 0) {
                if (!(L > 0.0) || !isfinite(l)) atomicOr(err, 1);
                if (site) site[p] = l;
            }
            contrib = a.patw[p] * l;
        }
        contrib = tile_sum<LPP>(contrib);
        if (lane == 0) part[tile] = contrib;
    }
}

// ---------------------------------------------------------------------------
// fused pre-order pass + branch-length gradient
// ---------------------------------------------------------------------------
// Pre-order partials are rescaled to a per-pattern maximum in [0.5, 1)
// (an exact power of two) after every op. The branch-length ratios do not
// depend on the scale of q, but the ratio's denominator q . (v_a o v_b) must
// stay inside the FP32 range: its states need not line up with q's maximum,
// so a q left small (a lazier rescaling) drove it below the smallest normal
// value on deep trees.
constexpr int kQRange = 0;
// Edges whose per-pattern gradient terms a warp buffers before summing them.
constexpr int kEdgeBuf = 16;

// Minimum resident blocks per SM the pre-order kernel is compiled for (by
// lane layout and element size; MINB > 0 overrides): one lane per pattern
// holds the four categories of q, both children's prefetched partials and
// the two outputs, in at most 168 registers in FP32 (three blocks, twelve
// warps per SM); FP64 needs twice the registers (two blocks).
template <typename T, int LPP>
struct PreMinBlocks {
    static constexpr int value = LPP == 1 ? (sizeof(T) == 8 ? 2 : 3) : 4;
};

// Fused pre-order pass and branch-length gradient. Per parent n with
// children a, b and category r (Sec. "Algorithmic advances", linear-time
// gradient): v_c = P_c p_c, u_a = q_n o v_b, u_b = q_n o v_a,
// q_c = P_c^T u_c, and the edge ratio u_c . (dP_c p_c) / u_c . v_c summed
// over categories with their weights (the denominator is the pattern
// likelihood up to the scales of q and p, so no scale bookkeeping). The
// categories are taken one at a time: each category's products are formed
// and consumed before the next one's, so only q_n, the children's partials
// and the two outputs stay live across the op. dP_c comes from shared
// memory for every child (a column for tip states), so any derivative of P
// (dP/dt, or dP/dtheta) takes the same path.
template <typename T, int LPP, int CPL, int NR, bool BATCH, int MINB>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, MINB > 0 ? MINB : PreMinBlocks<T, LPP>::value)
k_pre4(const DevPreOp* __restrict__ ops_, int n_ops_, const __grid_constant__ NucArgs<T> a_,
       const T* __restrict__ piw_, double* __restrict__ gpart_, const BatchRef<T> br) {
    constexpr int TP = 32 / LPP;
    constexpr bool kFull = NR > 0 && LPP * CPL == NR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = lane % LPP, pp = lane / LPP;
    const int R = NR > 0 ? NR : a_.R;
    const int cs = R * 4;  // matrix column stride (all categories of a column)
    V4<T>* slots = reinterpret_cast<V4<T>*>(smem_raw) + (size_t)warp * a_.n_slots * CPL * 32;
    unsigned char* pipe_base = reinterpret_cast<unsigned char*>(
        reinterpret_cast<V4<T>*>(smem_raw) + (size_t)kWarpsPerBlock * a_.n_slots * CPL * 32);
    WarpPipe<DevPreOp, T, 4> pipe;
    pipe.obuf = reinterpret_cast<DevPreOp*>(pipe_base + (size_t)warp * pipe_bytes<DevPreOp, T, 4>(R));
    pipe.mbuf = reinterpret_cast<T*>(pipe.obuf + 3);
    pipe.matf = kColStride * 4 * R;
    pipe.init(lane);
    BatchJob<T>* stage = reinterpret_cast<BatchJob<T>*>(
        pipe_base + (size_t)kWarpsPerBlock * pipe_bytes<DevPreOp, T, 4>(R)) + warp;
    // gradient terms of up to kEdgeBuf edges, [edge][lane] (row stride 33),
    // summed over the lanes kEdgeBuf edges at a time: one store per edge and
    // lane instead of a five-step shuffle reduction per edge
    T* gbuf = reinterpret_cast<T*>(reinterpret_cast<BatchJob<T>*>(
                  pipe_base + (size_t)kWarpsPerBlock * pipe_bytes<DevPreOp, T, 4>(R)) +
              kWarpsPerBlock) +
              (size_t)warp * kEdgeBuf * 33;
    const NucArgs<T>& a = pick_args<BATCH>(a_, stage);
    bool act[CPL];
#pragma unroll
    for (int j = 0; j < CPL; ++j) act[j] = kFull || (r0 + j * LPP < R);
    const V4<T> zero = {T(0), T(0), T(0), T(0)};
    const int nw = gridDim.x * kWarpsPerBlock;
    const DevPreOp* ops = ops_;
    int n_ops = n_ops_;
    double* gpart = gpart_;
    const T* piw = piw_;
    int cur = -1;
    for (int next = blockIdx.x * kWarpsPerBlock + warp; BATCH || next < a_.n_tiles; next += nw) {
        int tile = next;
        if constexpr (BATCH) {
            if (!batch_claim(br, a_.n_tiles, stage, cur, tile, lane)) break;
            ops = static_cast<const DevPreOp*>(stage->ops);
            n_ops = stage->n_ops;
            gpart = stage->gpart;
            piw = stage->piw;
        }
        const int p = tile * TP + pp;
        const size_t off0 = ((size_t)r0 * a.Ppad + p) * 4;
        const size_t offj = (size_t)LPP * a.Ppad * 4;
        const T wpt = (p < a.P) ? (T)a.patw[p] : T(0);
        int nbuf = 0, my_edge = 0;  // buffered edges; lane e holds edge e's row
        auto flush_edges = [&]() {
            __syncwarp();
            if (lane < nbuf) {
                T acc = T(0);
                for (int i = 0; i < 32; ++i) acc += gbuf[lane * 33 + i];
                gpart[(size_t)my_edge * a.n_tiles + tile] = (double)acc;
            }
            __syncwarp();
            nbuf = 0;
        };
        // a child's post-order partial (memory, or tip partials), prefetched
        // (a tip with states is read as matrix columns, its x left unset)
        auto child_x = [&](int child, int kind, V4<T>* x) {
            if (kind == kTipStates || kind < 0) {
#pragma unroll
                for (int j = 0; j < CPL; ++j) x[j] = zero;
                return;
            }
            const T* b = (kind == kTipPartials) ? a.tipbuf[child] : a.pool + (size_t)child * a.bstride;
#pragma unroll
            for (int j = 0; j < CPL; ++j) x[j] = act[j] ? ld4(b + off0 + j * offj) : zero;
        };
        // shared-memory matrices of op j: P of both children, and the
        // derivative of each child whose edge is listed
        auto issue_mats = [&](int j) {
            const DevPreOp& o = pipe.obuf[j % 3];
            const int idx[4] = {o.mat[0], o.mat[1], o.edge[0] >= 0 ? o.dmat[0] : -1,
                                o.edge[1] >= 0 ? o.dmat[1] : -1};
            pipe.issue_mats(j, n_ops, idx, a.mat, a.mat_stride, lane);
        };
        V4<T> prevq[CPL];  // the q output the next op reads from registers
#pragma unroll
        for (int j = 0; j < CPL; ++j) prevq[j] = zero;
        // inputs of the current op (A) and the next one (B, loaded while
        // the current op computes)
        int tsA[2], tsB[2];
        V4<T> xA[2][CPL], xB[2][CPL];
        {
            const int4 h = op_head(ops, 0, n_ops);
            tsA[0] = tip_state(a, h.x, h.z, p);
            tsA[1] = tip_state(a, h.y, h.w, p);
            child_x(h.x, h.z, xA[0]);
            child_x(h.y, h.w, xA[1]);
        }
        __syncwarp();
        pipe.issue_op(ops, 0, n_ops, lane);
        pipe.issue_op(ops, 1, n_ops, lane);
        cp_async_commit();
        cp_async_wait_all();
        __syncwarp();
        if (n_ops > 0) issue_mats(0);
        cp_async_commit();
        // one op: k's inputs in xc / tsc, k + 1's loaded into xn / tsn
        auto op_body = [&](int k, V4<T> (&xc)[2][CPL], V4<T> (&xn)[2][CPL], int (&tsc)[2],
                           int (&tsn)[2]) {
            cp_async_wait_all();
            __syncwarp();
            // op k + 1's inputs, first read by the next op, issued first
            // (children and kinds from the descriptor copy in shared memory,
            // not a global load whose result the addresses wait for)
            if (k + 1 < n_ops) {
                const DevPreOp& o1 = pipe.obuf[(k + 1) % 3];
                tsn[0] = tip_state(a, o1.child[0], o1.kind[0], p);
                tsn[1] = tip_state(a, o1.child[1], o1.kind[1], p);
                child_x(o1.child[0], o1.kind[0], xn[0]);
                child_x(o1.child[1], o1.kind[1], xn[1]);
            }
            pipe.issue_op(ops, k + 2, n_ops, lane);
            if (k + 1 < n_ops) issue_mats(k + 1);
            cp_async_commit();
            const DevPreOp& op = pipe.obuf[k % 3];
            const int kd0 = op.kind[0], kd1 = op.kind[1], qsrc = op.q_src;
            const bool e0 = op.edge[0] >= 0, e1 = op.edge[1] >= 0;
            const bool nq0 = op.need_q[0] != 0, nq1 = op.need_q[1] != 0;
            const T* mk = pipe.mats(k) + r0 * 4;
            const T* mP0 = mk;
            const T* mP1 = mk + pipe.matf;
            const T* mD0 = mk + 2 * pipe.matf;
            const T* mD1 = mk + 3 * pipe.matf;
            const int tc0 = tip_col((int8_t)tsc[0]) * cs, tc1 = tip_col((int8_t)tsc[1]) * cs;
            // q of the parent into prevq (from registers it is there already)
            if (qsrc == kFromRoot) {
                const V4<T> pv = ldg4(piw);
#pragma unroll
                for (int j = 0; j < CPL; ++j) prevq[j] = pv;
            } else if (qsrc >= 0) {
#pragma unroll
                for (int j = 0; j < CPL; ++j) prevq[j] = slots[(qsrc * CPL + j) * 32 + lane];
            } else if (qsrc == kFromMemory) {
                const T* qm = a.pool + (size_t)op.q_buf_in * a.bstride + off0;
#pragma unroll
                for (int j = 0; j < CPL; ++j) prevq[j] = act[j] ? ld4(qm + j * offj) : zero;
            }
            T den_l = T(0), num0 = T(0), num1 = T(0);
            V4<T> qa[CPL], qb[CPL];
            // the categories for one combination of child kinds: no branch
            // inside but the q of a tip (a derivative or internal q whose
            // result is not asked for is formed anyway and not used)
            auto categories = [&](auto tip0_c, auto tip1_c) {
                constexpr bool TIP0 = decltype(tip0_c)::value, TIP1 = decltype(tip1_c)::value;
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    // qa / qb of a tip are set only when asked for, and read
                    // only then
                    if (!act[j]) {
                        qa[j] = zero;
                        qb[j] = zero;
                        continue;
                    }
                    const int cj = j * LPP * 4;
                    const T wr = a.catw[r0 + j * LPP];
                    const V4<T> q = prevq[j];
                    // v_c = P_c p_c and dP_c p_c (columns of P and dP for a tip state).
                    // The scalar chain (matvec<T>, the same bits as the packed
                    // FP32 form): issued here it is faster than the packed form,
                    // whose broadcast operand pairs cost moves (2.47 -> 2.40 ms at
                    // 512 x 100k); the post-order kernel is faster packed.
                    const V4<T> v0 = TIP0 ? lds4(mP0 + tc0 + cj) : matvec<T>(mP0 + cj, cs, xc[0][j]);
                    const V4<T> v1 = TIP1 ? lds4(mP1 + tc1 + cj) : matvec<T>(mP1 + cj, cs, xc[1][j]);
                    const V4<T> u0 = mul(q, v1), u1 = mul(q, v0);
                    den_l += wr * dot(u0, v0);
                    const V4<T> d0 = TIP0 ? lds4(mD0 + tc0 + cj) : matvec<T>(mD0 + cj, cs, xc[0][j]);
                    const V4<T> d1 = TIP1 ? lds4(mD1 + tc1 + cj) : matvec<T>(mD1 + cj, cs, xc[1][j]);
                    num0 += wr * dot(u0, d0);
                    num1 += wr * dot(u1, d1);
                    // q of a tip only when it is asked for (materialised q)
                    if (!TIP0 || nq0) qa[j] = matTvec(mP0 + cj, cs, u0);
                    if (!TIP1 || nq1) qb[j] = matTvec(mP1 + cj, cs, u1);
                }
            };
            using yes = std::true_type;
            using no = std::false_type;
            if (kd0 == kTipStates) {
                if (kd1 == kTipStates) categories(yes{}, yes{});
                else categories(yes{}, no{});
            } else {
                if (kd1 == kTipStates) categories(no{}, yes{});
                else categories(no{}, no{});
            }
            if (e0 || e1) {
                // both children's ratios share it (FP32: the fast division, 2 ulp)
                const T wden = ratio_div(wpt, group_sum<LPP>(den_l));
                if (e0) {
                    const T num = group_sum<LPP>(num0);
                    gbuf[nbuf * 33 + lane] = (r0 == 0) ? num * wden : T(0);
                    if (lane == nbuf) my_edge = op.edge[0];
                    if (++nbuf == kEdgeBuf) flush_edges();
                }
                if (e1) {
                    const T num = group_sum<LPP>(num1);
                    gbuf[nbuf * 33 + lane] = (r0 == 0) ? num * wden : T(0);
                    if (lane == nbuf) my_edge = op.edge[1];
                    if (++nbuf == kEdgeBuf) flush_edges();
                }
            }
            // q outputs: rescaled when out of range, then to a slot, the
            // op's buffer and/or the registers the next op reads
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (!(c == 0 ? nq0 : nq1)) continue;
                V4<T>* qc = c == 0 ? qa : qb;
                T m = vmax_all<CPL>(qc);
#pragma unroll
                for (int o = 1; o < LPP; o <<= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
                const int e = frexp_exp(m);
                if (e < -kQRange || e > kQRange) scale_by_pow2(qc, CPL, -e);   // e != 0
                const int so = op.q_slot_out[c];
                if (so >= 0) {
#pragma unroll
                    for (int j = 0; j < CPL; ++j) slots[(so * CPL + j) * 32 + lane] = qc[j];
                }
                const int bo = op.q_buf_out[c];
                if (bo >= 0) {
                    T* b = a.pool + (size_t)bo * a.bstride + off0;
#pragma unroll
                    for (int j = 0; j < CPL; ++j)
                        if (act[j]) st4(b + j * offj, qc[j]);
                }
                if (op.q_reg == c) {
#pragma unroll
                    for (int j = 0; j < CPL; ++j) prevq[j] = qc[j];
                }
            }
        };
        // one call site: a second inlined copy of the op body costs registers
        // (it spilled, 3.96 against 2.44 ms at 512 x 100k) and could round
        // FP64 differently from the first (contractions are the compiler's
        // choice there), with the copy an op took depending on its position
        for (int k = 0; k < n_ops; ++k) {
            op_body(k, xA, xB, tsA, tsB);
            tsA[0] = tsB[0];
            tsA[1] = tsB[1];
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                xA[0][j] = xB[0][j];
                xA[1][j] = xB[1][j];
            }
        }
        if (nbuf > 0) flush_edges();
        cp_async_wait_all();
    }
}

// ---------------------------------------------------------------------------
// edge derivatives from stored pre- and post-order partials
// ---------------------------------------------------------------------------
template <typename T, int LPP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_edge4(const DevEdge* __restrict__ edges, int n_edges, NucArgs<T> a, const T* __restrict__ Qw,
        double* __restrict__ gpart) {
    constexpr int TP = 32 / LPP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane % LPP, pp = lane / LPP;
    const bool ract = r < a.R;
    const T wr = ract ? a.catw[r] : T(0);
    const T rr = ract ? a.rates[r] : T(0);
    const V4<T> q0 = ldg4(Qw), q1 = ldg4(Qw + 4), q2 = ldg4(Qw + 8), q3 = ldg4(Qw + 12);
    const int nw = gridDim.x * kWarpsPerBlock;
    for (int tile = blockIdx.x * kWarpsPerBlock + warp; tile < a.n_tiles; tile += nw) {
        const int p = tile * TP + pp;
        const size_t off = ((size_t)r * a.Ppad + p) * 4;
        const T wpt = (p < a.P) ? (T)a.patw[p] : T(0);
        for (int k = 0; k < n_edges; ++k) {
            const DevEdge e = edges[k];
            V4<T> x = {T(0), T(0), T(0), T(0)}, qq = {T(0), T(0), T(0), T(0)};
            if (e.kind == kTipStates) {
                const int s = a.tips[(size_t)e.post * a.Ppad + p];
                const bool amb = !(s >= 0 && s < 4);
                x = {T(amb || s == 0), T(amb || s == 1), T(amb || s == 2), T(amb || s == 3)};
            } else if (ract) {
                const T* b = (e.kind == kTipPartials) ? a.tipbuf[e.post]
                                                      : a.pool + (size_t)e.post * a.bstride;
                x = ld4(b + off);
            }
            if (ract) qq = ld4(a.pool + (size_t)e.pre * a.bstride + off);
            const V4<T> Qx = {dot(q0, x), dot(q1, x), dot(q2, x), dot(q3, x)};
            const T num = group_sum<LPP>(wr * rr * dot(qq, Qx));
            const T den = group_sum<LPP>(wr * dot(qq, x));
            T g = wpt * (num / den);
            g = tile_sum<LPP, T>(g);
            if (lane == 0) gpart[(size_t)e.edge * a.n_tiles + tile] = (double)g;
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// Lanes per pattern of the root and edge-derivative kernels (one category
// per lane).
int nuc_lanes(const Instance* I) {
    return I->R <= 1 ? 1 : I->R <= 2 ? 2 : I->R <= 4 ? 4 : 8;
}

// Lanes per pattern of the post- and pre-order kernels, as their dispatch
// instantiates them: with four categories 1 (all categories in one lane)
// unless TL_NUC_LANES selects 2 or 4; fewer categories use four lanes (one
// category each), more use eight. Tile counts (and so the columns of the
// gradient partials) follow from it.
int nuc_lanes_main(const Instance* I) {
    static int env = -1;
    if (env < 0) {
        const char* s = getenv("TL_NUC_LANES");
        env = s ? atoi(s) : 0;
    }
    if (I->R < 4) return 4;
    if (I->R > 4) return 8;
    return (env == 1 || env == 2 || env == 4) ? env : 1;
}

// Lanes per pattern of the pre-order kernel: with four categories
// TL_PRE_LANES (1, 2 or 4, at least the post-order kernel's), else the
// post-order kernel's.
int nuc_lanes_pre(const Instance* I) {
    static int env = -1;
    if (env < 0) {
        const char* s = getenv("TL_PRE_LANES");
        env = s ? atoi(s) : 0;
    }
    const int main = nuc_lanes_main(I);
    if (I->R != 4) return main;
    const int lpp = (env == 1 || env == 2 || env == 4) ? env : main;
    return std::max(lpp, main);
}

int nuc_cpl(const Instance* I) {
    const int lpp = nuc_lanes_main(I);
    return (I->R + lpp - 1) / lpp;
}

int nuc_tiles_for(const Instance* I, int lpp) { return I->Ppad / (32 / lpp); }
int nuc_tiles(const Instance* I) { return nuc_tiles_for(I, nuc_lanes(I)); }
int nuc_tiles_main(const Instance* I) { return nuc_tiles_for(I, nuc_lanes_main(I)); }
int nuc_tiles_pre(const Instance* I) { return nuc_tiles_for(I, nuc_lanes_pre(I)); }

// Patterns per lane of the post-order kernel: 2 (TL_POST_PPL=1 for one)
// with one lane per pattern and four categories, else 1.
int nuc_post_ppl(const Instance* I) {
    static int env = -1;
    if (env < 0) {
        const char* s = getenv("TL_POST_PPL");
        env = s ? atoi(s) : 2;
    }
    return (env == 2 && nuc_lanes_main(I) == 1 && I->R == 4) ? 2 : 1;
}

int nuc_smem_per_slot(const Instance* I) {
    return 32 * (nuc_cpl(I) * 4 * I->elt + (int)sizeof(int));
}

template <typename T>
static NucArgs<T> make_args(const Instance* I, int n_slots) {
    NucArgs<T> a;
    a.pool = reinterpret_cast<T*>(I->pool);
    a.epool = I->scale_pool;
    a.tips = I->tip_pool;
    a.tipbuf = reinterpret_cast<T* const*>(I->d_buf);
    a.mat = reinterpret_cast<const T*>(I->d_matw);
    a.patw = I->d_patw;
    a.bstride = (size_t)I->R * I->Ppad * 4;
    a.P = I->P;
    a.Ppad = I->Ppad;
    a.R = I->R;
    a.n_slots = n_slots;
    a.rescale = I->rescale;
    a.mat_stride = (int)I->matw_stride;
    a.n_tiles = nuc_tiles(I);  // launchers of the main kernels override
    for (int r = 0; r < kMaxCat; ++r) {
        a.catw[r] = (T)(r < I->R ? I->h_catw[r] : 0.0);
        a.rates[r] = (T)(r < I->R ? I->h_rates[r] : 0.0);
    }
    return a;
}

// Persistent grid: as many blocks as fit at once, never more than the tiles.
template <typename K>
static int grid_for(const Instance* I, K kernel, size_t smem, int n_tiles) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarpsPerBlock * 32, smem);
    const int need = (n_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int fit = std::max(1, per_sm) * std::max(1, sms);
    return std::max(1, std::min(need, fit));
}

#define TL_NUC_DISPATCH(I, FN, ...)                                      \
    do {                                                                 \
        const int lpp_ = nuc_lanes(I);                                   \
        if ((I)->prec == kF32) {                                         \
            if (lpp_ == 1) FN<float, 1>(__VA_ARGS__);                    \
            else if (lpp_ == 2) FN<float, 2>(__VA_ARGS__);               \
            else if (lpp_ == 4) FN<float, 4>(__VA_ARGS__);               \
            else FN<float, 8>(__VA_ARGS__);                              \
        } else {                                                         \
            if (lpp_ == 1) FN<double, 1>(__VA_ARGS__);                   \
            else if (lpp_ == 2) FN<double, 2>(__VA_ARGS__);              \
            else if (lpp_ == 4) FN<double, 4>(__VA_ARGS__);              \
            else FN<double, 8>(__VA_ARGS__);                             \
        }                                                                \
    } while (0)

// Four categories (the common case) get kernels specialised on the count
// and on the lane layout; other counts use a runtime-R kernel.
#define TL_MAIN_DISPATCH_T(T, I, FN, ...)                                   \
    do {                                                                    \
        const int lpp_ = nuc_lanes_main(I);                                 \
        if ((I)->R == 4) {                                                  \
            if (lpp_ == 1) FN<T, 1, 4, 4>(__VA_ARGS__);                     \
            else if (lpp_ == 2) FN<T, 2, 2, 4>(__VA_ARGS__);                \
            else FN<T, 4, 1, 4>(__VA_ARGS__);                               \
        } else if ((I)->R < 4) {                                            \
            FN<T, 4, 1, 0>(__VA_ARGS__);                                    \
        } else {                                                            \
            FN<T, 8, 1, 0>(__VA_ARGS__);                                    \
        }                                                                   \
    } while (0)
// The same over the pre-order kernel's lane layouts.
#define TL_PRE_DISPATCH_T(T, I, FN, ...)                                    \
    do {                                                                    \
        const int lpp_ = nuc_lanes_pre(I);                                  \
        if ((I)->R == 4) {                                                  \
            if (lpp_ == 1) FN<T, 1, 4, 4>(__VA_ARGS__);                     \
            else if (lpp_ == 2) FN<T, 2, 2, 4>(__VA_ARGS__);                \
            else FN<T, 4, 1, 4>(__VA_ARGS__);                               \
        } else if ((I)->R < 4) {                                            \
            FN<T, 4, 1, 0>(__VA_ARGS__);                                    \
        } else {                                                            \
            FN<T, 8, 1, 0>(__VA_ARGS__);                                    \
        }                                                                   \
    } while (0)
#define TL_MAIN_DISPATCH(I, FN, ...)                                        \
    do {                                                                    \
        if ((I)->prec == kF32) TL_MAIN_DISPATCH_T(float, I, FN, __VA_ARGS__); \
        else TL_MAIN_DISPATCH_T(double, I, FN, __VA_ARGS__);               \
    } while (0)

template <typename T, int LPP, int CPL, int NR, int PPL>
static void post4_tp(Instance* I, const DevPostOp* d_ops, int n_ops, int n_slots) {
    const size_t smem = (size_t)kWarpsPerBlock *
                        (n_slots * nuc_smem_per_slot(I) * PPL + pipe_bytes<DevPostOp, T, 2>(I->R));
    cudaFuncSetAttribute(k_post4<T, LPP, CPL, NR, false, PPL>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    NucArgs<T> a = make_args<T>(I, n_slots);
    a.n_tiles = nuc_tiles_for(I, LPP) / PPL;
    const int grid = grid_for(I, k_post4<T, LPP, CPL, NR, false, PPL>, smem, a.n_tiles);
    k_post4<T, LPP, CPL, NR, false, PPL><<<grid, kWarpsPerBlock * 32, smem, I->stream>>>(
        d_ops, n_ops, a, BatchRef<T>{});
}

template <typename T, int LPP, int CPL, int NR>
static void post4_t(Instance* I, const DevPostOp* d_ops, int n_ops, int n_slots) {
    if constexpr (LPP == 1 && NR == 4) {
        if (nuc_post_ppl(I) == 2) return post4_tp<T, LPP, CPL, NR, 2>(I, d_ops, n_ops, n_slots);
    }
    post4_tp<T, LPP, CPL, NR, 1>(I, d_ops, n_ops, n_slots);
}

int launch_post4(Instance* I, const DevPostOp* d_ops, int n_ops, int n_slots) {
    TL_MAIN_DISPATCH(I, post4_t, I, d_ops, n_ops, n_slots);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "post-order kernel");
}

template <typename T, int LPP>
static void root4_t(Instance* I, int kind, int root, const double* pi, double* d_site,
                    double* d_part) {
    const int grid = grid_for(I, k_root4<T, LPP, false>, 0, nuc_tiles(I));
    k_root4<T, LPP, false><<<grid, kWarpsPerBlock * 32, 0, I->stream>>>(
        kind, root, make_args<T>(I, 0), pi, d_site, d_part, I->d_err + 1, BatchRef<T>{});
}

int launch_root4(Instance* I, int root_kind, int root, int model, double* d_site,
                 double* d_part) {
    TL_NUC_DISPATCH(I, root4_t, I, root_kind, root, I->models[model].pi, d_site, d_part);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "root kernel");
}

// Register budget of the one-lane-per-pattern pre-order kernel: TL_PRE_MINB
// = 3 or 4 compiles it for three or four resident blocks per SM.
static int pre_minb() {
    static int env = -1;
    if (env < 0) {
        const char* s = getenv("TL_PRE_MINB");
        env = s ? atoi(s) : 0;
    }
    return env;
}

// Dynamic shared memory of a pre-order block: per warp its q slots, the
// op/matrix pipeline, a batch job copy and the edge-term buffer.
template <typename T>
static size_t pre4_smem(const Instance* I, int n_slots, int cpl) {
    return (size_t)kWarpsPerBlock * ((size_t)n_slots * cpl * 32 * 4 * sizeof(T) +
                                     pipe_bytes<DevPreOp, T, 4>(I->R) + sizeof(BatchJob<T>) +
                                     kEdgeBuf * 33 * sizeof(T));
}

// q slots the pre-order planner may use: as many as leave room for
// 228 KB / (the blocks per SM the kernel is compiled for) of shared memory
// per block, at most 12.
int nuc_pre_slot_cap(const Instance* I) {
    const int lpp = nuc_lanes_pre(I), cpl = (I->R + lpp - 1) / lpp;
    int blocks = lpp == 1 ? (I->elt == 8 ? 2 : 3) : 4;
    if (lpp == 1 && I->R == 4 && I->prec == kF32 && pre_minb() == 4) blocks = 4;
    const size_t fixed = I->prec == kF32 ? pre4_smem<float>(I, 0, cpl) : pre4_smem<double>(I, 0, cpl);
    const size_t per = (size_t)kWarpsPerBlock * cpl * 32 * 4 * I->elt;
    const size_t budget = (size_t)228 * 1024 / blocks;
    if (budget <= fixed) return 0;
    return (int)std::min<size_t>(12, (budget - fixed) / per);
}

template <typename T, int LPP, int CPL, int NR, int MINB>
static void pre4_tm(Instance* I, const DevPreOp* d_ops, int n_ops, int n_slots, const void* piw,
                    double* d_gpart) {
    const size_t smem = pre4_smem<T>(I, n_slots, CPL);
    auto kern = k_pre4<T, LPP, CPL, NR, false, MINB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    NucArgs<T> a = make_args<T>(I, n_slots);
    a.n_tiles = nuc_tiles_for(I, LPP);
    const int grid = grid_for(I, kern, smem, a.n_tiles);
    kern<<<grid, kWarpsPerBlock * 32, smem, I->stream>>>(
        d_ops, n_ops, a, reinterpret_cast<const T*>(piw), d_gpart, BatchRef<T>{});
}

template <typename T, int LPP, int CPL, int NR>
static void pre4_t(Instance* I, const DevPreOp* d_ops, int n_ops, int n_slots, const void* piw,
                   double* d_gpart) {
    if constexpr (LPP == 1 && NR == 4 && sizeof(T) == 4) {
        if (pre_minb() == 3) return pre4_tm<T, LPP, CPL, NR, 3>(I, d_ops, n_ops, n_slots, piw, d_gpart);
        if (pre_minb() == 4) return pre4_tm<T, LPP, CPL, NR, 4>(I, d_ops, n_ops, n_slots, piw, d_gpart);
    }
    pre4_tm<T, LPP, CPL, NR, 0>(I, d_ops, n_ops, n_slots, piw, d_gpart);
}

// dgen: the derivative slots hold any derivative of P (dP/dtheta); the
// kernel reads every child's derivative matrix, so both cases take one path
int launch_pre4(Instance* I, const DevPreOp* d_ops, int n_ops, int n_slots, int model,
                double* d_gpart, int dgen) {
    (void)dgen;
    if (I->prec == kF32)
        TL_PRE_DISPATCH_T(float, I, pre4_t, I, d_ops, n_ops, n_slots, I->models[model].piw,
                          d_gpart);
    else
        TL_PRE_DISPATCH_T(double, I, pre4_t, I, d_ops, n_ops, n_slots, I->models[model].piw,
                          d_gpart);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "pre-order kernel");
}

template <typename T, int LPP>
static void edge4_t(Instance* I, const DevEdge* d_edges, int n_edges, const void* Qw,
                    double* d_gpart) {
    const int grid = grid_for(I, k_edge4<T, LPP>, 0, nuc_tiles(I));
    k_edge4<T, LPP><<<grid, kWarpsPerBlock * 32, 0, I->stream>>>(
        d_edges, n_edges, make_args<T>(I, 0), reinterpret_cast<const T*>(Qw), d_gpart);
}

int launch_edge4(Instance* I, const DevEdge* d_edges, int n_edges, int model, double* d_gpart) {
    TL_NUC_DISPATCH(I, edge4_t, I, d_edges, n_edges, I->models[model].Qw, d_gpart);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "edge-derivative kernel");
}


// ---------------------------------------------------------------------------
// batched launchers: one job table upload and one launch for n instances of
// one precision and category count
// ---------------------------------------------------------------------------
// Table layout in the batch area: [counter, pad x3][tile_begin: n + 1 ints,
// padded to 16 bytes][jobs].
template <typename T>
static int upload_table(Batch* B, int which, const std::vector<BatchJob<T>>& jobs,
                        const std::vector<int>& begin, BatchRef<T>* br) {
    const int n = (int)jobs.size();
    const size_t hdr = 16 + (((size_t)(n + 1) * sizeof(int) + 15) / 16) * 16;
    std::vector<unsigned char> buf(hdr + (size_t)n * sizeof(BatchJob<T>), 0);
    std::memcpy(buf.data() + 16, begin.data(), sizeof(int) * (n + 1));
    std::memcpy(buf.data() + hdr, jobs.data(), sizeof(BatchJob<T>) * n);
    void* d = nullptr;
    int rc = batch_upload(B, which, buf.data(), buf.size(), &d);
    if (rc) return rc;
    unsigned char* base = static_cast<unsigned char*>(d);
    br->counter = reinterpret_cast<int*>(base);
    br->tile_begin = reinterpret_cast<const int*>(base + 16);
    br->jobs = reinterpret_cast<const BatchJob<T>*>(base + hdr);
    br->n_jobs = n;
    return TL_OK;
}

// Jobs in order of decreasing op count (stable), so the longest tile walks
// are claimed first; jobs without ops or tiles are left out.
static std::vector<int> by_work(const int* n_ops, int n) {
    std::vector<int> order;
    for (int k = 0; k < n; ++k)
        if (n_ops[k] > 0) order.push_back(k);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return n_ops[x] > n_ops[y]; });
    return order;
}

template <typename T, int LPP, int CPL, int NR, int PPL>
static int post4_batch_tp(Batch* B, Instance* const* I, const DevPostOp* const* d_ops,
                          const int* n_ops, const int* n_slots, int n) {
    const std::vector<int> order = by_work(n_ops, n);
    if (order.empty()) return TL_OK;
    std::vector<BatchJob<T>> jobs;
    std::vector<int> begin(1, 0);
    int max_slots = 0;
    long long total = 0;
    for (int k : order) {
        BatchJob<T> j{};
        j.a = make_args<T>(I[k], n_slots[k]);
        j.a.n_tiles = nuc_tiles_for(I[k], LPP) / PPL;
        j.ops = d_ops[k];
        j.n_ops = n_ops[k];
        jobs.push_back(j);
        total += j.a.n_tiles;
        if (total > (1LL << 30)) return batch_fail(B, TL_ERR_UNSUPPORTED, "batch too large");
        begin.push_back((int)total);
        max_slots = std::max(max_slots, n_slots[k]);
    }
    BatchRef<T> br;
    int rc = upload_table(B, 0, jobs, begin, &br);
    if (rc) return rc;
    Instance* I0 = I[order[0]];
    const size_t smem = (size_t)kWarpsPerBlock *
                        (max_slots * nuc_smem_per_slot(I0) * PPL +
                         pipe_bytes<DevPostOp, T, 2>(I0->R) + sizeof(BatchJob<T>));
    cudaFuncSetAttribute(k_post4<T, LPP, CPL, NR, true, PPL>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    NucArgs<T> layout = make_args<T>(I0, max_slots);
    layout.n_tiles = (int)total;
    const int grid = grid_for(I0, k_post4<T, LPP, CPL, NR, true, PPL>, smem, (int)total);
    k_post4<T, LPP, CPL, NR, true, PPL><<<grid, kWarpsPerBlock * 32, smem, B->stream>>>(
        nullptr, 0, layout, br);
    B->launches += 1;
    return batch_cuda(B, cudaGetLastError(), "batched post-order kernel");
}

template <typename T, int LPP, int CPL, int NR>
static int post4_batch_t(Batch* B, Instance* const* I, const DevPostOp* const* d_ops,
                         const int* n_ops, const int* n_slots, int n) {
    if constexpr (LPP == 1 && NR == 4) {
        if (nuc_post_ppl(I[0]) == 2)
            return post4_batch_tp<T, LPP, CPL, NR, 2>(B, I, d_ops, n_ops, n_slots, n);
    }
    return post4_batch_tp<T, LPP, CPL, NR, 1>(B, I, d_ops, n_ops, n_slots, n);
}

#define TL_BATCH_DISPATCH(I0, FN, ...)                                          \
    do {                                                                        \
        if ((I0)->prec == kF32) TL_MAIN_DISPATCH_T(float, I0, return FN, __VA_ARGS__); \
        else TL_MAIN_DISPATCH_T(double, I0, return FN, __VA_ARGS__);           \
    } while (0)

int nuc_batch_post(Batch* B, Instance* const* I, const DevPostOp* const* d_ops, const int* n_ops,
                   const int* n_slots, int n) {
    if (n <= 0) return TL_OK;
    TL_BATCH_DISPATCH(I[0], post4_batch_t, B, I, d_ops, n_ops, n_slots, n);
    return TL_OK;
}

template <typename T, int LPP>
static int root4_batch_t(Batch* B, Instance* const* I, const int* kind, const int* root,
                         const int* model, int n, double* const* d_part) {
    std::vector<BatchJob<T>> jobs;
    std::vector<int> begin(1, 0);
    long long total = 0;
    for (int k = 0; k < n; ++k) {
        BatchJob<T> j{};
        j.a = make_args<T>(I[k], 0);
        j.a.n_tiles = nuc_tiles_for(I[k], LPP);
        j.root_kind = kind[k];
        j.root = root[k];
        j.pi = I[k]->models[model[k]].pi;
        j.part = d_part[k];
        j.err = I[k]->d_err + 1;
        jobs.push_back(j);
        total += j.a.n_tiles;
        if (total > (1LL << 30)) return batch_fail(B, TL_ERR_UNSUPPORTED, "batch too large");
        begin.push_back((int)total);
    }
    BatchRef<T> br;
    int rc = upload_table(B, 1, jobs, begin, &br);
    if (rc) return rc;
    NucArgs<T> layout = make_args<T>(I[0], 0);
    layout.n_tiles = (int)total;
    const int grid = grid_for(I[0], k_root4<T, LPP, true>, 0, (int)total);
    k_root4<T, LPP, true><<<grid, kWarpsPerBlock * 32, 0, B->stream>>>(
        0, 0, layout, nullptr, nullptr, nullptr, nullptr, br);
    B->launches += 1;
    return batch_cuda(B, cudaGetLastError(), "batched root kernel");
}

int nuc_batch_root(Batch* B, Instance* const* I, const int* kind, const int* root,
                   const int* model, int n, double* const* d_part) {
    if (n <= 0) return TL_OK;
    const int lpp = nuc_lanes(I[0]);
    if (I[0]->prec == kF32) {
        if (lpp == 1) return root4_batch_t<float, 1>(B, I, kind, root, model, n, d_part);
        if (lpp == 2) return root4_batch_t<float, 2>(B, I, kind, root, model, n, d_part);
        if (lpp == 4) return root4_batch_t<float, 4>(B, I, kind, root, model, n, d_part);
        return root4_batch_t<float, 8>(B, I, kind, root, model, n, d_part);
    }
    if (lpp == 1) return root4_batch_t<double, 1>(B, I, kind, root, model, n, d_part);
    if (lpp == 2) return root4_batch_t<double, 2>(B, I, kind, root, model, n, d_part);
    if (lpp == 4) return root4_batch_t<double, 4>(B, I, kind, root, model, n, d_part);
    return root4_batch_t<double, 8>(B, I, kind, root, model, n, d_part);
}

template <typename T, int LPP, int CPL, int NR>
static int pre4_batch_t(Batch* B, Instance* const* I, const DevPreOp* const* d_ops,
                        const int* n_ops, const int* n_slots, const int* model,
                        double* const* d_gpart, int n) {
    const std::vector<int> order = by_work(n_ops, n);
    if (order.empty()) return TL_OK;
    std::vector<BatchJob<T>> jobs;
    std::vector<int> begin(1, 0);
    int max_slots = 0;
    long long total = 0;
    for (int k : order) {
        BatchJob<T> j{};
        j.a = make_args<T>(I[k], n_slots[k]);
        j.a.n_tiles = nuc_tiles_for(I[k], LPP);
        j.ops = d_ops[k];
        j.n_ops = n_ops[k];
        j.piw = reinterpret_cast<const T*>(I[k]->models[model[k]].piw);
        j.Qw = reinterpret_cast<const T*>(I[k]->models[model[k]].Qw);
        j.gpart = d_gpart[k];
        jobs.push_back(j);
        total += j.a.n_tiles;
        if (total > (1LL << 30)) return batch_fail(B, TL_ERR_UNSUPPORTED, "batch too large");
        begin.push_back((int)total);
        max_slots = std::max(max_slots, n_slots[k]);
    }
    BatchRef<T> br;
    int rc = upload_table(B, 2, jobs, begin, &br);
    if (rc) return rc;
    Instance* I0 = I[order[0]];
    const size_t smem = pre4_smem<T>(I0, max_slots, CPL);
    cudaFuncSetAttribute(k_pre4<T, LPP, CPL, NR, true, 0>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    NucArgs<T> layout = make_args<T>(I0, max_slots);
    layout.n_tiles = (int)total;
    const int grid = grid_for(I0, k_pre4<T, LPP, CPL, NR, true, 0>, smem, (int)total);
    k_pre4<T, LPP, CPL, NR, true, 0><<<grid, kWarpsPerBlock * 32, smem, B->stream>>>(
        nullptr, 0, layout, nullptr, nullptr, br);
    B->launches += 1;
    return batch_cuda(B, cudaGetLastError(), "batched pre-order kernel");
}

int nuc_batch_pre(Batch* B, Instance* const* I, const DevPreOp* const* d_ops, const int* n_ops,
                  const int* n_slots, const int* model, double* const* d_gpart, int n) {
    if (n <= 0) return TL_OK;
    if (I[0]->prec == kF32)
        TL_PRE_DISPATCH_T(float, I[0], return pre4_batch_t, B, I, d_ops, n_ops, n_slots, model,
                          d_gpart, n);
    else
        TL_PRE_DISPATCH_T(double, I[0], return pre4_batch_t, B, I, d_ops, n_ops, n_slots, model,
                          d_gpart, n);
    return TL_OK;
}

}  // namespace tl
