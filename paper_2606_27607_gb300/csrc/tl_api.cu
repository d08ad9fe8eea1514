// C ABI of the treelik library: instance lifecycle, input validation, the
// host-side scheduler that turns an operation list into a device walk (op
// reordering and on-chip slot assignment), launches, and fixed-order
// reductions. Every numerical step runs in the kernels of tl_model.cu,
// tl_nuc.cu and tl_generic.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "tl_internal.cuh"

namespace tl {

static thread_local std::string g_create_err;

// Round an FP32 value to TF32 (10 explicit mantissa bits), nearest with ties
// away from zero, as cvt.rna.tf32.f32 does on the device.
float tf32_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float y;
    std::memcpy(&y, &u, 4);
    return y;
}

int fail(Instance* I, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (I) I->err = buf;
    else g_create_err = buf;
    return code;
}

int cuda_check(Instance* I, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TL_OK;
    return fail(I, e == cudaErrorMemoryAllocation ? TL_ERR_OOM : TL_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

// Fixed-order sum of n doubles by one warp: lane l adds in[l], in[l + 32],
// ... in order, then a butterfly over the lanes (every lane gets the sum).
// Single and batched reductions both use it, so their results are identical.
__device__ __forceinline__ double warp_row_sum(const double* __restrict__ in, int n) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) acc += in[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

constexpr int kRedWarps = 8;  // rows per block of the reductions

// Sum each of n_out rows of n_in doubles in a fixed order (deterministic).
__global__ void k_reduce_rows(const double* __restrict__ in, int n_in, int n_out,
                              double* __restrict__ out) {
    const int row = blockIdx.x * kRedWarps + (threadIdx.x >> 5);
    if (row >= n_out) return;
    const double v = warp_row_sum(in + (size_t)row * n_in, n_in);
    if ((threadIdx.x & 31) == 0) out[row] = v;
}

// Batched form over RedJob descriptors: global row -> job by binary search
// over row_begin; jobs[j] owns rows [row_begin[j], row_begin[j + 1]).
__global__ void k_reduce_batch(const RedJob* __restrict__ jobs, const int* __restrict__ row_begin,
                               int n_jobs, int total) {
    const int row = blockIdx.x * kRedWarps + (threadIdx.x >> 5);
    if (row >= total) return;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_begin[mid] <= row) lo = mid;
        else hi = mid - 1;
    }
    const RedJob J = jobs[lo];
    const int g = row - row_begin[lo];
    const int src = J.inv ? J.inv[g] : g;
    const double v = src >= 0 ? warp_row_sum(J.in + (size_t)src * J.n_in, J.n_in) : 0.0;
    if ((threadIdx.x & 31) == 0) J.out[g] = v;
}

// out[map[k]] = in[k] for k < n; out has n_out entries, the rest zeroed.
__global__ void k_scatter(const double* __restrict__ in, const int* __restrict__ map, int n,
                          double* __restrict__ out, int n_out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_out; i += gridDim.x * blockDim.x)
        out[i] = 0.0;
    __syncthreads();
    // single block launch: the zeroing above is complete for this block
    for (int k = threadIdx.x; k < n; k += blockDim.x) out[map[k]] = in[k];
}

int reduce_fixed(Instance* I, const double* d_in, int n_out, int n_in, double* d_out) {
    if (n_out <= 0) return TL_OK;
    k_reduce_rows<<<(n_out + kRedWarps - 1) / kRedWarps, kRedWarps * 32, 0, I->stream>>>(
        d_in, n_in, n_out, d_out);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "reduction");
}

}  // namespace tl

using namespace tl;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
namespace {

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// instance's stream) from the device's default pool, which is told to keep
// freed memory: creating and destroying instances (a server admitting and
// evicting them) then reuses memory without synchronising the device.
void keep_pool_memory(int dev) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    done.push_back(dev);
}

template <typename P>
int dev_alloc(Instance* I, P** p, size_t bytes, const char* what) {
    keep_pool_memory(I->device);
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, bytes ? bytes : 16, I->stream);
    if (e == cudaErrorMemoryAllocation) {
        // the pool may hold freed blocks too small or too scattered for this
        // request: let every pending free complete, return unused memory to
        // the device and try once more
        cudaGetLastError();
        cudaDeviceSynchronize();
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, I->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
        e = cudaMallocAsync(&q, bytes ? bytes : 16, I->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(I, TL_ERR_OOM, "device allocation of %zu bytes for %s failed: %s", bytes,
                    what, cudaGetErrorString(e));
    }
    I->bytes += bytes;
    *p = reinterpret_cast<P*>(q);
    return TL_OK;
}

// Stream-ordered free: work already queued on the instance's stream finishes
// with the memory first; batched calls make each instance's stream wait for
// them, so their uses are covered too.
void dev_free(Instance* I, void* p) {
    if (p) cudaFreeAsync(p, I->stream);
}

int ensure_scratch(Instance* I, size_t doubles) {
    if (I->red_cap >= doubles) return TL_OK;
    if (I->d_red) {
        dev_free(I, I->d_red);
        I->bytes -= I->red_cap * sizeof(double);
        I->d_red = nullptr;
        I->red_cap = 0;
    }
    size_t cap = std::max<size_t>(doubles, 1 << 16);
    int rc = dev_alloc(I, &I->d_red, cap * sizeof(double), "reduction scratch");
    if (rc) return rc;
    I->red_cap = cap;
    return TL_OK;
}

// Pinned host staging ring for small uploads: a slot is reused only after
// the copy that last read it has completed (its event), so callers' host
// arrays are free as soon as a call returns and no copy waits on the stream.
struct PinnedSlot {
    void* h = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
};
constexpr int kRing = 8;

// Page-locked staging buffers outlive their instances: a destroyed
// instance's ring slots (buffer and event) go to a process-wide list that
// new instances draw from, so admission and eviction do not pay for
// page-locked allocations. A slot's event guards its reuse as before.
std::mutex g_pinned_mu;
std::vector<PinnedSlot> g_pinned;
constexpr size_t kPinnedKeep = 4096;

void take_pinned(PinnedSlot* s) {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    if (g_pinned.empty()) return;
    *s = g_pinned.back();
    g_pinned.pop_back();
}

void give_pinned(PinnedSlot& s) {
    if (!s.h && !s.ev) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    if (g_pinned.size() < kPinnedKeep && s.h) {
        g_pinned.push_back(s);
    } else {
        if (s.ev) cudaEventSynchronize(s.ev);
        if (s.h) cudaFreeHost(s.h);
        if (s.ev) cudaEventDestroy(s.ev);
    }
    s = PinnedSlot();
}

// Upload bytes to op area `which` unless identical to the last upload.
struct OpArea {
    void* d = nullptr;
    size_t cap = 0;
    std::vector<char> last;
};

int h2d(Instance* I, void* dst, const void* src, size_t bytes);

int upload(Instance* I, OpArea& A, const void* src, size_t bytes, void** dptr) {
    if (bytes == 0) {
        *dptr = A.d;
        return TL_OK;
    }
    if (A.last.size() == bytes && std::memcmp(A.last.data(), src, bytes) == 0 && A.d) {
        *dptr = A.d;
        return TL_OK;
    }
    if (A.cap < bytes) {
        if (A.d) {
            dev_free(I, A.d);
            I->bytes -= A.cap;
        }
        size_t cap = std::max<size_t>(bytes * 2, 4096);
        int rc = dev_alloc(I, &A.d, cap, "op list");
        if (rc) return rc;
        A.cap = cap;
        A.last.clear();
    }
    int rc = h2d(I, A.d, src, bytes);
    if (rc) return rc;
    A.last.assign((const char*)src, (const char*)src + bytes);
    *dptr = A.d;
    return TL_OK;
}

struct Extra {
    PinnedSlot ring[kRing];
    int ring_next = 0;
    OpArea areas[6];
    cudaEvent_t order_ev = nullptr;  // orders this stream against a batch stream
    // double-buffered tip states (tl_set_tip_states_all_async): pool[i] and
    // the events ordering each copy against the kernels that read the pool
    int8_t* tip_pools[2] = {nullptr, nullptr};
    int tip_active = 0;              // the pool I->tip_pool points to
    int tip_pending = -1;            // a pool being filled for the next call
    cudaStream_t tip_stream = nullptr;
    cudaEvent_t tip_copied[2] = {nullptr, nullptr};   // copy into pool i done
    cudaEvent_t tip_free[2] = {nullptr, nullptr};     // last kernel reading pool i done
    std::vector<void*> gen_q;     // generic path: scratch pre-order buffers
    double* d_out = nullptr;      // small result area
    size_t out_cap = 0;
};

Extra& extra(Instance* I) {
    return *reinterpret_cast<Extra*>(I->host_extra);
}

// Copy `bytes` from host `src` to device `dst` on the instance stream through
// the pinned ring.
int h2d(Instance* I, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return TL_OK;
    Extra& X = extra(I);
    PinnedSlot& s = X.ring[X.ring_next];
    X.ring_next = (X.ring_next + 1) % kRing;
    if (!s.h && !s.ev) take_pinned(&s);  // a slot (and its event) from the shared list
    cudaError_t e = cudaSuccess;
    if (s.ev) e = cudaEventSynchronize(s.ev);
    else e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_check(I, e, "staging event");
    if (s.cap < bytes) {
        if (s.h) cudaFreeHost(s.h);
        s.cap = std::max<size_t>(bytes, 64 * 1024);
        e = cudaHostAlloc(&s.h, s.cap, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            s.h = nullptr;
            s.cap = 0;
            return cuda_check(I, e, "pinned staging");
        }
    }
    std::memcpy(s.h, src, bytes);
    e = cudaMemcpyAsync(dst, s.h, bytes, cudaMemcpyHostToDevice, I->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.ev, I->stream);
    return cuda_check(I, e, "host to device copy");
}

int ensure_out(Instance* I, size_t n) {
    Extra& X = extra(I);
    if (X.out_cap >= n) return TL_OK;
    if (X.d_out) {
        dev_free(I, X.d_out);
        I->bytes -= X.out_cap * sizeof(double);
    }
    size_t cap = std::max<size_t>(n, 4096);
    int rc = dev_alloc(I, &X.d_out, cap * sizeof(double), "result area");
    if (rc) return rc;
    X.out_cap = cap;
    return TL_OK;
}

bool use_nuc(const Instance* I) { return I->S == 4 && (I->prec == kF32 || I->prec == kF64); }
bool use_tc(const Instance* I) { return I->prec == kTF32; }

// Device area `which` with at least `bytes` (contents not kept).
void* area(Instance* I, int which, size_t bytes, int* rc) {
    OpArea& A = extra(I).areas[which];
    if (A.cap < bytes) {
        if (A.d) {
            dev_free(I, A.d);
            I->bytes -= A.cap;
            A.d = nullptr;
        }
        const size_t cap = std::max<size_t>(bytes * 2, 4096);
        if ((*rc = dev_alloc(I, &A.d, cap, "op list"))) return nullptr;
        A.cap = cap;
    }
    A.last.clear();
    *rc = TL_OK;
    return A.d;
}

int max_slots(const Instance* I) {
    // keep the per-block on-chip slot area near 56 KB so four blocks
    // (sixteen warps) stay resident per SM
    const int per = nuc_smem_per_slot(I) * kWarpsPerBlock;
    return std::max(0, std::min(12, (56 * 1024) / per));
}

int check_numeric_flag(Instance* I) {
    int h[3] = {0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, I->d_err, 3 * sizeof(int), cudaMemcpyDeviceToHost, I->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
    if (e != cudaSuccess) return cuda_check(I, e, "error flag");
    if (h[2]) {
        cudaMemsetAsync(I->d_err + 2, 0, sizeof(int), I->stream);
        return fail(I, TL_ERR_TIMEOUT, "a tensor-core kernel wait gave up (code 0x%x: bits 0-2 "
                    "empty/full/done barrier, bits 8-10 post/pre1/pre2 kernel, bit 11 adjoint)", h[2]);
    }
    if (h[0] || h[1]) {
        cudaMemsetAsync(I->d_err, 0, 2 * sizeof(int), I->stream);
        if (h[0])
            return fail(I, TL_ERR_NUMERIC, "model set-up failed on the device (check %d: "
                        "non-positive frequency, zero mean rate or Jacobi did not converge)", h[0]);
        return fail(I, TL_ERR_NUMERIC, "a pattern likelihood is zero, negative or not finite");
    }
    return TL_OK;
}

#define CHECK_INST(I)                                                        \
    do {                                                                     \
        if (!(I)) return fail(nullptr, TL_ERR_ARG, "null instance");         \
    } while (0)

// -------- post-order scheduling ---------------------------------------------
struct PostPlan {
    std::vector<DevPostOp> dev;
    int n_slots = 0;
};

int plan_post(Instance* I, const tl_op* ops, int n, PostPlan* plan, bool dry) {
    const int NB = I->n_bufs;
    std::vector<int> producer(NB, -1);
    std::vector<int> consumers(n, 0);
    std::vector<int> first_read(NB, n);
    std::vector<int> writer(NB, -1);
    for (int k = 0; k < n; ++k)
        if (ops[k].dest >= 0 && ops[k].dest < NB && writer[ops[k].dest] < 0) writer[ops[k].dest] = k;
    for (int k = 0; k < n; ++k) {
        const tl_op& o = ops[k];
        const int ch[2] = {o.child1, o.child2};
        const int mt[2] = {o.mat1, o.mat2};
        if (o.dest < I->n_tips || o.dest >= NB)
            return fail(I, TL_ERR_INDEX, "op %d: dest %d is not an internal buffer", k, o.dest);
        for (int c = 0; c < 2; ++c) {
            if (ch[c] < 0 || ch[c] >= NB)
                return fail(I, TL_ERR_INDEX, "op %d: child %d out of range", k, ch[c]);
            if (mt[c] < 0 || mt[c] >= I->n_mats)
                return fail(I, TL_ERR_INDEX, "op %d: matrix %d out of range", k, mt[c]);
            if (!I->mat_set[mt[c]])
                return fail(I, TL_ERR_STATE, "op %d: matrix %d not computed", k, mt[c]);
            if (ch[c] == o.dest)
                return fail(I, TL_ERR_ORDER, "op %d: dest is also a child", k);
            if (writer[ch[c]] > k)
                return fail(I, TL_ERR_ORDER, "op %d: buffer %d is read before op %d writes it", k,
                            ch[c], writer[ch[c]]);
            if (ch[c] < I->n_tips) {
                if (!I->tip_set[ch[c]])
                    return fail(I, TL_ERR_STATE, "op %d: tip %d has no data", k, ch[c]);
            } else if (producer[ch[c]] < 0 && !I->buf_written[ch[c] - I->n_tips]) {
                return fail(I, TL_ERR_STATE, "op %d: buffer %d read before it is written", k, ch[c]);
            }
            first_read[ch[c]] = std::min(first_read[ch[c]], k);
            if (producer[ch[c]] >= 0) consumers[producer[ch[c]]]++;
        }
        if (producer[o.dest] >= 0)
            return fail(I, TL_ERR_ORDER, "op %d: buffer %d written twice", k, o.dest);
        if (first_read[o.dest] < k)
            return fail(I, TL_ERR_ORDER, "op %d: buffer %d read by op %d before it is written", k,
                        o.dest, first_read[o.dest]);
        producer[o.dest] = k;
    }
    if (dry) return TL_OK;

    // Sethi-Ullman order: evaluate the child subtree needing more slots
    // first. Only for forests (each local result consumed once).
    bool forest = true;
    for (int k = 0; k < n; ++k)
        if (consumers[k] > 1) forest = false;
    std::vector<int> order;
    order.reserve(n);
    std::vector<int> need(n, 1);
    auto local = [&](int k, int c) {
        int ch = c == 0 ? ops[k].child1 : ops[k].child2;
        return (ch >= I->n_tips) ? producer[ch] : -1;
    };
    if (forest) {
        for (int k = 0; k < n; ++k) {
            int x = local(k, 0), y = local(k, 1);
            if (x >= 0 && y >= 0)
                need[k] = need[x] == need[y] ? need[x] + 1 : std::max(need[x], need[y]);
            else if (x >= 0 || y >= 0)
                need[k] = need[x >= 0 ? x : y];
        }
        std::vector<char> emitted(n, 0);
        // iterative guard against deep recursion on caterpillars
        for (int k = 0; k < n; ++k) {
            if (consumers[k] == 0) {
                // explicit stack version of emit
                std::vector<std::pair<int, int>> st;
                st.push_back({k, 0});
                while (!st.empty()) {
                    auto& [v, phase] = st.back();
                    int x = local(v, 0), y = local(v, 1);
                    if (x >= 0 && y >= 0 && need[y] > need[x]) std::swap(x, y);
                    if (phase == 0) {
                        phase = 1;
                        if (x >= 0) { st.push_back({x, 0}); continue; }
                    }
                    if (phase == 1) {
                        phase = 2;
                        if (y >= 0) { st.push_back({y, 0}); continue; }
                    }
                    order.push_back(v);
                    emitted[v] = 1;
                    st.pop_back();
                }
            }
        }
        if ((int)order.size() != n) {  // should not happen; fall back
            order.clear();
            for (int k = 0; k < n; ++k) order.push_back(k);
        }
    } else {
        for (int k = 0; k < n; ++k) order.push_back(k);
    }

    // The op just before hands its result over in registers when it is the
    // only consumer; other in-list results get a shared-memory slot by linear
    // scan (or are re-read from memory when no slot is free).
    std::vector<int> pos(n), sole_consumer(n, -1);
    for (int idx = 0; idx < n; ++idx) pos[order[idx]] = idx;
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < 2; ++c) {
            int pk = local(k, c);
            if (pk >= 0 && consumers[pk] == 1) sole_consumer[pk] = k;
        }
    const int cap = max_slots(I) / (use_nuc(I) ? nuc_post_ppl(I) : 1);
    std::vector<int> slot_of(n, -1), remaining(n, 0);
    for (int k = 0; k < n; ++k) remaining[k] = consumers[k];
    std::vector<int> free_slots;
    for (int s = cap - 1; s >= 0; --s) free_slots.push_back(s);
    int used = 0;
    plan->dev.resize(n);
    for (int idx = 0; idx < n; ++idx) {
        const int k = order[idx];
        const tl_op& o = ops[k];
        DevPostOp d;
        std::memset(&d, 0, sizeof d);
        const int ch[2] = {o.child1, o.child2};
        const int mt[2] = {o.mat1, o.mat2};
        for (int c = 0; c < 2; ++c) {
            d.mat[c] = mt[c];
            if (ch[c] < I->n_tips) {
                d.kind[c] = I->tip_set[ch[c]] == 1 ? kTipStates : kTipPartials;
                d.child[c] = ch[c];
            } else {
                d.kind[c] = kInternal;
                d.child[c] = ch[c] - I->n_tips;
            }
            const int pk = local(k, c);
            if (pk >= 0 && idx > 0 && order[idx - 1] == pk) d.slot_in[c] = kFromRegisters;
            else d.slot_in[c] = (pk >= 0 && slot_of[pk] >= 0) ? slot_of[pk] : kFromMemory;
        }
        for (int c = 0; c < 2; ++c) {
            int pk = local(k, c);
            if (pk >= 0 && --remaining[pk] == 0 && slot_of[pk] >= 0) free_slots.push_back(slot_of[pk]);
        }
        d.dest = o.dest - I->n_tips;
        d.slot_out = -1;
        const bool next_only = sole_consumer[k] >= 0 && pos[sole_consumer[k]] == idx + 1;
        if (consumers[k] > 0 && !next_only && !free_slots.empty()) {
            d.slot_out = free_slots.back();
            free_slots.pop_back();
            slot_of[k] = d.slot_out;
            used = std::max(used, d.slot_out + 1);
        }
        d.store = 1;
        plan->dev[idx] = d;
    }
    plan->n_slots = used;
    return TL_OK;
}

// -------- pre-order scheduling ----------------------------------------------
struct PrePlan {
    std::vector<DevPreOp> dev;
    int n_slots = 0;
    std::vector<int> edge_map;   // compact row -> user edge index
    std::vector<int> stored;     // pool indices of q written to memory
};

int plan_pre(Instance* I, const tl_pre_op* ops, int n, int n_grad, bool store_all,
             PrePlan* plan) {
    const int NB = I->n_bufs;
    std::vector<int> prod_op(NB, -1), prod_c(NB, -1);
    std::vector<int> child_op(2 * n, -1);   // op consuming output c of op k
    std::vector<int> edge_row(std::max(n_grad, 1), -1);
    plan->edge_map.clear();
    plan->stored.clear();
    for (int k = 0; k < n; ++k) {
        const tl_pre_op& o = ops[k];
        if (o.parent_pre != -1) {
            if (o.parent_pre < I->n_tips || o.parent_pre >= NB)
                return fail(I, TL_ERR_INDEX, "pre op %d: parent_pre %d not an internal buffer", k,
                            o.parent_pre);
            int j = prod_op[o.parent_pre];
            if (j >= 0) {
                if (child_op[2 * j + prod_c[o.parent_pre]] >= 0)
                    return fail(I, TL_ERR_ORDER, "pre op %d: q buffer %d consumed twice", k,
                                o.parent_pre);
                child_op[2 * j + prod_c[o.parent_pre]] = k;
            } else if (!I->buf_written[o.parent_pre - I->n_tips]) {
                return fail(I, TL_ERR_STATE, "pre op %d: parent_pre %d holds no data", k,
                            o.parent_pre);
            }
        }
        for (int c = 0; c < 2; ++c) {
            if (o.child[c] < 0 || o.child[c] >= NB)
                return fail(I, TL_ERR_INDEX, "pre op %d: child %d out of range", k, o.child[c]);
            if (o.child[c] < I->n_tips ? !I->tip_set[o.child[c]]
                                       : !I->buf_written[o.child[c] - I->n_tips])
                return fail(I, TL_ERR_STATE, "pre op %d: child %d holds no data", k, o.child[c]);
            if (o.mat[c] < 0 || o.mat[c] >= I->n_mats || !I->mat_set[o.mat[c]])
                return fail(I, TL_ERR_INDEX, "pre op %d: matrix %d not available", k, o.mat[c]);
            if (o.dmat[c] >= I->n_mats || (o.dmat[c] >= 0 && !I->mat_set[o.dmat[c]]))
                return fail(I, TL_ERR_INDEX, "pre op %d: dmat %d not available", k, o.dmat[c]);
            if (o.edge[c] >= 0) {
                if (o.edge[c] >= n_grad)
                    return fail(I, TL_ERR_INDEX, "pre op %d: edge %d >= n_grad", k, o.edge[c]);
                if (o.dmat[c] < 0)
                    return fail(I, TL_ERR_ARG, "pre op %d: edge requested without dmat", k);
                if (edge_row[o.edge[c]] >= 0)
                    return fail(I, TL_ERR_ORDER, "pre op %d: edge %d requested twice", k, o.edge[c]);
                edge_row[o.edge[c]] = (int)plan->edge_map.size();
                plan->edge_map.push_back(o.edge[c]);
            }
            if (o.pre[c] >= 0) {
                if (o.pre[c] < I->n_tips || o.pre[c] >= NB)
                    return fail(I, TL_ERR_INDEX, "pre op %d: pre %d not an internal buffer", k,
                                o.pre[c]);
                if (prod_op[o.pre[c]] >= 0)
                    return fail(I, TL_ERR_ORDER, "pre op %d: pre buffer %d written twice", k,
                                o.pre[c]);
                prod_op[o.pre[c]] = k;
                prod_c[o.pre[c]] = c;
            }
        }
    }
    // a pre-order output may not overwrite a post-order child of this list
    // (children are prefetched ahead of the ops that write q)
    {
        std::vector<char> is_child(NB, 0);
        for (int k = 0; k < n; ++k)
            for (int c = 0; c < 2; ++c) is_child[ops[k].child[c]] = 1;
        for (int k = 0; k < n; ++k)
            for (int c = 0; c < 2; ++c)
                if (ops[k].pre[c] >= 0 && is_child[ops[k].pre[c]])
                    return fail(I, TL_ERR_ORDER, "pre op %d: pre buffer %d is also a child", k,
                                ops[k].pre[c]);
    }
    // order: depth first from each root op, smaller-need subtree first
    std::vector<int> need(n, 0), parent_op(n, -1);
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < 2; ++c)
            if (child_op[2 * k + c] >= 0) parent_op[child_op[2 * k + c]] = k;
    for (int k = n - 1; k >= 0; --k) {
        int x = child_op[2 * k], y = child_op[2 * k + 1];
        if (x >= 0 && y >= 0) {
            int a = std::min(need[x], need[y]), b = std::max(need[x], need[y]);
            need[k] = std::max(2, std::max(a + 1, b));
        } else if (x >= 0 || y >= 0) {
            need[k] = std::max(1, need[x >= 0 ? x : y]);
        }
    }
    std::vector<int> order;
    order.reserve(n);
    for (int k = 0; k < n; ++k) {
        if (parent_op[k] >= 0) continue;
        std::vector<int> st{k};
        while (!st.empty()) {
            int v = st.back();
            st.pop_back();
            order.push_back(v);
            int x = child_op[2 * v], y = child_op[2 * v + 1];
            // push larger-need first so the smaller one is processed first
            if (x >= 0 && y >= 0) {
                if (need[x] < need[y]) std::swap(x, y);
                st.push_back(x);
                st.push_back(y);
            } else if (x >= 0) {
                st.push_back(x);
            } else if (y >= 0) {
                st.push_back(y);
            }
        }
    }
    if ((int)order.size() != n) return fail(I, TL_ERR_ORDER, "pre-order op list is not a forest");
    // parents must precede children in the given list too (validated above by
    // prod_op lookups happening in list order)
    const int cap = use_nuc(I) ? nuc_pre_slot_cap(I) : 0;
    std::vector<int> free_slots;
    for (int s = cap - 1; s >= 0; --s) free_slots.push_back(s);
    std::vector<int> q_slot(2 * n, -1), pos(n);
    for (int idx = 0; idx < n; ++idx) pos[order[idx]] = idx;
    int used = 0;
    plan->dev.resize(n);
    for (int idx = 0; idx < n; ++idx) {
        const int k = order[idx];
        const tl_pre_op& o = ops[k];
        DevPreOp d;
        std::memset(&d, 0, sizeof d);
        d.q_buf_in = -1;
        d.q_reg = -1;
        if (o.parent_pre == -1) {
            d.q_src = kFromRoot;
        } else {
            const int j = prod_op[o.parent_pre];
            const int c = j >= 0 ? prod_c[o.parent_pre] : 0;
            if (j >= 0 && pos[j] == idx - 1 && use_nuc(I)) {
                d.q_src = kFromRegisters;
            } else if (j >= 0 && q_slot[2 * j + c] >= 0) {
                d.q_src = q_slot[2 * j + c];
                free_slots.push_back(d.q_src);
            } else {
                d.q_src = kFromMemory;
                d.q_buf_in = o.parent_pre - I->n_tips;
            }
        }
        for (int c = 0; c < 2; ++c) {
            if (o.child[c] < I->n_tips) {
                d.kind[c] = I->tip_set[o.child[c]] == 1 ? kTipStates : kTipPartials;
                d.child[c] = o.child[c];
            } else {
                d.kind[c] = kInternal;
                d.child[c] = o.child[c] - I->n_tips;
            }
            d.mat[c] = o.mat[c];
            d.dmat[c] = o.dmat[c];
            d.edge[c] = o.edge[c] >= 0 ? edge_row[o.edge[c]] : -1;
            d.q_slot_out[c] = -1;
            d.q_buf_out[c] = -1;
            const int cons = child_op[2 * k + c];
            if (o.pre[c] >= 0) {
                // a named q is kept on chip when a later op of this list
                // consumes it, and written to its buffer otherwise (a later
                // call reads it) or when every q is to be stored
                d.need_q[c] = 1;
                const bool next = cons >= 0 && pos[cons] == idx + 1;
                if (next) d.q_reg = c;  // the next op takes q_c from registers
                if (store_all || cons < 0) {
                    d.q_buf_out[c] = o.pre[c] - I->n_tips;
                } else if (next) {
                    // registers only
                } else if (!free_slots.empty()) {
                    d.q_slot_out[c] = free_slots.back();
                    free_slots.pop_back();
                    q_slot[2 * k + c] = d.q_slot_out[c];
                    used = std::max(used, d.q_slot_out[c] + 1);
                } else {
                    d.q_buf_out[c] = o.pre[c] - I->n_tips;
                }
                if (d.q_buf_out[c] >= 0) plan->stored.push_back(o.pre[c]);
            }
        }
        plan->dev[idx] = d;
    }
    plan->n_slots = used;
    return TL_OK;
}

// A pool filled by tl_set_tip_states_all_async becomes the instance's tip
// pool at the next call that launches work: the instance stream waits for
// the copy, and the pool it leaves is marked free once the work queued so
// far (the last readers of that pool) is done.
int activate_tip_pool(Instance* I) {
    Extra& X = extra(I);
    if (X.tip_pending < 0) return TL_OK;
    const int nxt = X.tip_pending, old = X.tip_active;
    X.tip_pending = -1;
    cudaError_t e = cudaStreamWaitEvent(I->stream, X.tip_copied[nxt], 0);
    if (e == cudaSuccess) e = cudaEventRecord(X.tip_free[old], I->stream);
    if (e != cudaSuccess) return cuda_check(I, e, "tip pool switch");
    X.tip_active = nxt;
    I->tip_pool = X.tip_pools[nxt];
    for (int t = 0; t < I->n_tips; ++t) {
        I->h_tipst[t] = I->tip_pool + (size_t)t * I->Ppad;
        I->h_buf[t] = nullptr;
        I->tip_set[t] = 1;
    }
    int rc;
    if ((rc = h2d(I, I->d_tipst, I->h_tipst.data(), sizeof(int8_t*) * I->n_tips))) return rc;
    return h2d(I, I->d_buf, I->h_buf.data(), sizeof(void*) * I->n_tips);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int tl_last_error(const tl_instance* inst, char* buf, size_t len) {
    if (!buf || len == 0) return TL_ERR_ARG;
    const std::string& s = inst ? reinterpret_cast<const Instance*>(inst)->err : g_create_err;
    size_t n = std::min(len - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
    return TL_OK;
}

int tl_device_bytes(const tl_instance* inst, size_t* out) {
    if (!inst || !out) return TL_ERR_ARG;
    *out = reinterpret_cast<const Instance*>(inst)->bytes;
    return TL_OK;
}

int tl_destroy(tl_instance* inst) {
    if (!inst) return TL_ERR_ARG;
    Instance* I = reinterpret_cast<Instance*>(inst);
    // nothing waits here: every free is ordered after the work queued on the
    // instance's stream, and the staging buffers go back to the shared list
    auto fr = [I](void* p) { dev_free(I, p); };
    fr(I->pool);
    fr(I->scale_pool);
    if (I->prec != kTF32)
        for (void* p : I->tip_part) fr(p);
    fr(I->tip_pool);
    fr(I->d_buf);
    fr(I->d_scale);
    fr(I->d_tipst);
    fr(I->d_patw);
    fr(I->d_mat64);
    fr(I->d_matw);
    for (ModelDev& M : I->models) {
        fr(M.Q);
        fr(M.pi);
        fr(M.V);
        fr(M.Vinv);
        fr(M.Vdf);
        fr(M.Vinvdf);
        fr(M.lam);
        fr(M.dQ);
        fr(M.G);
        fr(M.piw);
        fr(M.Qw);
        fr(M.pairs);
        fr(M.mu);
    }
    fr(I->d_red);
    fr(I->d_err);
    fr(I->d_rowsum);
    fr(I->tc_tip_pool);
    fr(I->d_tmp);
    if (I->host_extra) {
        Extra* X = reinterpret_cast<Extra*>(I->host_extra);
        for (auto& s : X->ring) give_pinned(s);
        for (auto& A : X->areas) fr(A.d);
        if (X->order_ev) cudaEventDestroy(X->order_ev);
        if (X->tip_stream) {
            cudaStreamSynchronize(X->tip_stream);
            cudaStreamDestroy(X->tip_stream);
        }
        for (int i = 0; i < 2; ++i) {
            if (X->tip_pools[i] && X->tip_pools[i] != I->tip_pool) fr(X->tip_pools[i]);
            if (X->tip_copied[i]) cudaEventDestroy(X->tip_copied[i]);
            if (X->tip_free[i]) cudaEventDestroy(X->tip_free[i]);
        }
        for (void* p : X->gen_q) fr(p);
        fr(X->d_out);
        delete X;
    }
    delete[] I->h_catw;
    delete[] I->h_rates;
    delete I;
    return TL_OK;
}

int tl_create(int n_tips, int n_patterns, int n_states, int n_categories, int n_buffers,
              int n_matrices, int n_models, unsigned flags, void* stream, tl_instance** out) {
    if (!out) return fail(nullptr, TL_ERR_ARG, "out is null");
    *out = nullptr;
    const unsigned precs = flags & (TL_PREC_F64 | TL_PREC_F32 | TL_PREC_TF32 | TL_PREC_BF16X3);
    if (precs == 0 || (precs & (precs - 1)))
        return fail(nullptr, TL_ERR_ARG, "exactly one TL_PREC_* flag is required");
    if (n_tips < 2 || n_patterns < 1 || n_states < 2 || n_states > kMaxStates ||
        n_categories < 1 || n_categories > kMaxCat || n_buffers < 1 || n_matrices < 1 ||
        n_models < 1)
        return fail(nullptr, TL_ERR_ARG,
                    "bad sizes (tips>=2, patterns>=1, 2<=states<=64, 1<=categories<=8, "
                    "buffers, matrices, models >= 1)");
    Prec prec = (precs == TL_PREC_F64) ? kF64 : (precs == TL_PREC_F32) ? kF32
                : (precs == TL_PREC_TF32) ? kTF32 : kBF16X3;
    if (prec == kF32 && n_states != 4)
        return fail(nullptr, TL_ERR_UNSUPPORTED, "TL_PREC_F32 is built for 4 states");
    if (prec == kBF16X3)
        return fail(nullptr, TL_ERR_UNSUPPORTED, "TL_PREC_BF16X3 is not built in this library");
    if (prec == kTF32 && (n_states < 5 || n_states > 64))
        return fail(nullptr, TL_ERR_UNSUPPORTED, "TL_PREC_TF32 is built for 5..64 states");
    // the tensor-core kernels hold both children's products of every
    // category in the 512 TMEM columns (2 x R x 64)
    if (prec == kTF32 && n_categories > 4)
        return fail(nullptr, TL_ERR_UNSUPPORTED, "TL_PREC_TF32 is built for at most 4 categories");
    if ((flags & TL_SCALE_NONE) && prec != kF64)
        return fail(nullptr, TL_ERR_ARG, "TL_SCALE_NONE needs TL_PREC_F64");
    if ((flags & TL_SPLIT_MATRICES) && prec != kTF32)
        return fail(nullptr, TL_ERR_ARG, "TL_SPLIT_MATRICES needs TL_PREC_TF32");
    if ((flags & TL_SPLIT_PARTIALS) && !(flags & TL_SPLIT_MATRICES))
        return fail(nullptr, TL_ERR_ARG, "TL_SPLIT_PARTIALS needs TL_PREC_TF32 | TL_SPLIT_MATRICES");

    Instance* I = new Instance();
    I->n_tips = n_tips;
    I->P = n_patterns;
    const int pad = (prec == kTF32 || prec == kBF16X3) ? 128 : kPadPatterns;
    I->Ppad = ((n_patterns + pad - 1) / pad) * pad;
    I->S = n_states;
    I->Spad = (n_states == 4) ? 4 : ((n_states + 3) / 4) * 4;
    if (prec == kTF32 || prec == kBF16X3) I->Spad = 64;
    I->R = n_categories;
    I->n_buffers = n_buffers;
    I->n_bufs = n_tips + n_buffers;
    I->n_mats = n_matrices;
    I->n_models = n_models;
    I->flags = flags;
    I->prec = prec;
    I->elt = (prec == kF64) ? 8 : 4;
    I->rescale = (flags & TL_SCALE_NONE) ? 0 : 1;
    I->split = (flags & TL_SPLIT_MATRICES) ? 1 : 0;
    I->split_partials = (flags & TL_SPLIT_PARTIALS) ? 1 : 0;
    I->stream = reinterpret_cast<cudaStream_t>(stream);
    I->h_catw = new double[kMaxCat];
    I->h_rates = new double[kMaxCat];
    for (int r = 0; r < kMaxCat; ++r) {
        I->h_catw[r] = r < n_categories ? 1.0 / n_categories : 0.0;
        I->h_rates[r] = r < n_categories ? 1.0 : 0.0;
    }
    I->host_extra = new Extra();
    cudaGetDevice(&I->device);

    auto bail = [&](int rc) {
        g_create_err = I->err;
        tl_destroy(reinterpret_cast<tl_instance*>(I));
        return rc;
    };
    int rc;
    const size_t nbuf_elems = (size_t)I->R * I->Ppad * I->Spad;
    if ((rc = dev_alloc(I, &I->pool, nbuf_elems * I->elt * n_buffers, "partials"))) return bail(rc);
    if ((rc = dev_alloc(I, &I->scale_pool, sizeof(int) * (size_t)I->Ppad * n_buffers, "scales")))
        return bail(rc);
    cudaMemsetAsync(I->scale_pool, 0, sizeof(int) * (size_t)I->Ppad * n_buffers, I->stream);
    if ((rc = dev_alloc(I, &I->d_buf, sizeof(void*) * I->n_bufs, "buffer table"))) return bail(rc);
    if ((rc = dev_alloc(I, &I->d_scale, sizeof(int*) * I->n_bufs, "scale table"))) return bail(rc);
    if ((rc = dev_alloc(I, &I->d_tipst, sizeof(int8_t*) * n_tips, "tip table"))) return bail(rc);
    I->h_buf.assign(I->n_bufs, nullptr);
    I->h_scale.assign(I->n_bufs, nullptr);
    I->h_tipst.assign(n_tips, nullptr);
    I->tip_part.assign(n_tips, nullptr);
    if ((rc = dev_alloc(I, &I->tip_pool, (size_t)n_tips * I->Ppad, "tip states"))) return bail(rc);
    cudaMemsetAsync(I->tip_pool, 0xff, (size_t)n_tips * I->Ppad, I->stream);
    I->tip_set.assign(n_tips, 0);
    I->buf_written.assign(n_buffers, 0);
    for (int b = 0; b < n_buffers; ++b) {
        I->h_buf[n_tips + b] = (char*)I->pool + nbuf_elems * I->elt * b;
        I->h_scale[n_tips + b] = I->scale_pool + (size_t)I->Ppad * b;
    }
    // staged through the page-locked ring: nothing here waits for the stream
    if ((rc = h2d(I, I->d_buf, I->h_buf.data(), sizeof(void*) * I->n_bufs)) ||
        (rc = h2d(I, I->d_scale, I->h_scale.data(), sizeof(int*) * I->n_bufs)) ||
        (rc = h2d(I, I->d_tipst, I->h_tipst.data(), sizeof(int8_t*) * n_tips)))
        return bail(rc);
    if ((rc = dev_alloc(I, &I->d_patw, sizeof(double) * I->Ppad, "pattern weights"))) return bail(rc);
    {
        std::vector<double> w(I->Ppad, 0.0);
        for (int p = 0; p < n_patterns; ++p) w[p] = 1.0;
        if ((rc = h2d(I, I->d_patw, w.data(), sizeof(double) * I->Ppad))) return bail(rc);
    }
    const size_t mat64 = (size_t)I->R * I->Spad * I->Spad;
    if ((rc = dev_alloc(I, &I->d_mat64, sizeof(double) * mat64 * n_matrices, "matrices")))
        return bail(rc);
    if (use_nuc(I)) I->matw_stride = (size_t)I->R * kColStride * 4;
    else if (prec == kTF32)
        I->matw_stride = (size_t)(I->split ? 4 : 2) * I->R * I->Spad * I->Spad;
    else I->matw_stride = (size_t)I->R * (I->Spad + 1) * I->Spad;
    const size_t matw_elems = prec == kTF32 ? tc_matw_floats(I) : I->matw_stride * n_matrices;
    if ((rc = dev_alloc(I, &I->d_matw, (size_t)I->elt * matw_elems, "matrix copies")))
        return bail(rc);
    I->mat_set.assign(n_matrices, 0);
    I->mat_len.assign(n_matrices, 0.0);
    I->mat_model.assign(n_matrices, -1);
    I->models.resize(n_models);
    const size_t SS = (size_t)I->Spad * I->Spad;
    for (ModelDev& M : I->models) {
        if ((rc = dev_alloc(I, &M.Q, sizeof(double) * SS, "Q")) ||
            (rc = dev_alloc(I, &M.pi, sizeof(double) * I->Spad, "pi")) ||
            (rc = dev_alloc(I, &M.V, sizeof(double) * SS, "V")) ||
            (rc = dev_alloc(I, &M.Vinv, sizeof(double) * SS, "Vinv")) ||
            (rc = dev_alloc(I, &M.lam, sizeof(double) * I->Spad, "lambda")) ||
            (rc = dev_alloc(I, &M.dQ, sizeof(double) * SS * kMaxDq, "dQ")) ||
            (rc = dev_alloc(I, &M.G, sizeof(double) * SS * kMaxDq * 2, "parameter basis")) ||
            (rc = dev_alloc(I, &M.piw, (size_t)I->elt * I->Spad, "pi copy")) ||
            (rc = dev_alloc(I, &M.Qw, (size_t)I->elt * SS, "Q copy")) ||
            (rc = dev_alloc(I, &M.pairs, sizeof(int) * 2 * TL_GY94_PAIRS, "pair table")) ||
            (rc = dev_alloc(I, &M.mu, sizeof(double), "mean rate")))
            return bail(rc);
        if (prec != kF64 &&
            ((rc = dev_alloc(I, &M.Vdf, 2 * sizeof(float) * SS, "V pairs")) ||
             (rc = dev_alloc(I, &M.Vinvdf, 2 * sizeof(float) * SS, "Vinv pairs"))))
            return bail(rc);
    }
    if (prec == kTF32) {
        if ((rc = dev_alloc(I, &I->d_rowsum, sizeof(float) * (size_t)n_matrices * I->R * I->Spad,
                            "row sums")))
            return bail(rc);
        if ((rc = tc_setup(I))) return bail(rc);
    }
    if ((rc = dev_alloc(I, &I->d_err, sizeof(int) * 4, "error flags"))) return bail(rc);
    cudaMemsetAsync(I->d_err, 0, sizeof(int) * 4, I->stream);
    I->tmp_cap = 4096;
    if ((rc = dev_alloc(I, &I->d_tmp, sizeof(double) * I->tmp_cap, "staging"))) return bail(rc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bail(cuda_check(I, e, "tl_create"));
    *out = reinterpret_cast<tl_instance*>(I);
    return TL_OK;
}

int tl_sync(tl_instance* inst) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    cudaError_t e = cudaStreamSynchronize(I->stream);
    if (e != cudaSuccess) return cuda_check(I, e, "tl_sync");
    return check_numeric_flag(I);
}

int tl_set_tip_states(tl_instance* inst, int tip, const int8_t* states) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (tip < 0 || tip >= I->n_tips) return fail(I, TL_ERR_INDEX, "tip %d out of range", tip);
    if (!states) return fail(I, TL_ERR_ARG, "states is null");
    int rc = activate_tip_pool(I);
    if (rc) return rc;
    int8_t* dst = I->tip_pool + (size_t)tip * I->Ppad;
    rc = h2d(I, dst, states, (size_t)I->P);
    if (rc) return rc;
    if (I->h_tipst[tip] != dst || I->h_buf[tip] != nullptr) {
        I->h_tipst[tip] = dst;
        I->h_buf[tip] = nullptr;
        if ((rc = h2d(I, I->d_tipst + tip, &I->h_tipst[tip], sizeof(int8_t*)))) return rc;
        if ((rc = h2d(I, I->d_buf + tip, &I->h_buf[tip], sizeof(void*)))) return rc;
    }
    I->tip_set[tip] = 1;
    return TL_OK;
}

int tl_set_tip_states_all_async(tl_instance* inst, const int8_t* states) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (!states) return fail(I, TL_ERR_ARG, "states is null");
    Extra& X = extra(I);
    cudaError_t e = cudaSuccess;
    if (!X.tip_stream) {
        e = cudaStreamCreateWithFlags(&X.tip_stream, cudaStreamNonBlocking);
        for (int i = 0; e == cudaSuccess && i < 2; ++i) {
            e = cudaEventCreateWithFlags(&X.tip_copied[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&X.tip_free[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_check(I, e, "tl_set_tip_states_all_async set-up");
        X.tip_pools[0] = I->tip_pool;
        X.tip_active = 0;
        // nothing has read the second pool yet
        if ((e = cudaEventRecord(X.tip_free[1], X.tip_stream)) != cudaSuccess)
            return cuda_check(I, e, "tl_set_tip_states_all_async set-up");
    }
    if (!X.tip_pools[1]) {
        int rc = dev_alloc(I, reinterpret_cast<void**>(&X.tip_pools[1]), (size_t)I->n_tips * I->Ppad,
                           "second tip pool");
        if (rc) return rc;
        // padding patterns read as ambiguous, as in the first pool
        e = cudaMemsetAsync(X.tip_pools[1], 0xff, (size_t)I->n_tips * I->Ppad, I->stream);
        if (e == cudaSuccess) e = cudaEventRecord(X.tip_free[1], I->stream);
        if (e != cudaSuccess) return cuda_check(I, e, "second tip pool");
    }
    // fill the pool that is neither active nor already pending
    const int tgt = X.tip_pending >= 0 ? X.tip_pending : 1 - X.tip_active;
    e = cudaStreamWaitEvent(X.tip_stream, X.tip_free[tgt], 0);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(X.tip_pools[tgt], I->Ppad, states, I->P, I->P, I->n_tips,
                              cudaMemcpyHostToDevice, X.tip_stream);
    if (e == cudaSuccess) e = cudaEventRecord(X.tip_copied[tgt], X.tip_stream);
    if (e != cudaSuccess) return cuda_check(I, e, "tl_set_tip_states_all_async");
    X.tip_pending = tgt;
    return TL_OK;
}

int tl_set_tip_states_all(tl_instance* inst, const int8_t* states) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (!states) return fail(I, TL_ERR_ARG, "states is null");
    int rc0 = activate_tip_pool(I);   // a pending asynchronous upload is superseded
    if (rc0) return rc0;
    cudaError_t e = cudaMemcpy2DAsync(I->tip_pool, I->Ppad, states, I->P, I->P, I->n_tips,
                                      cudaMemcpyHostToDevice, I->stream);
    if (e != cudaSuccess) return cuda_check(I, e, "tl_set_tip_states_all");
    bool changed = false;
    for (int t = 0; t < I->n_tips; ++t) {
        int8_t* dst = I->tip_pool + (size_t)t * I->Ppad;
        if (I->h_tipst[t] != dst || I->h_buf[t] != nullptr) changed = true;
        I->h_tipst[t] = dst;
        I->h_buf[t] = nullptr;
        I->tip_set[t] = 1;
    }
    int rc;
    if (changed) {
        if ((rc = h2d(I, I->d_tipst, I->h_tipst.data(), sizeof(int8_t*) * I->n_tips))) return rc;
        if ((rc = h2d(I, I->d_buf, I->h_buf.data(), sizeof(void*) * I->n_tips))) return rc;
    }
    return cuda_check(I, cudaStreamSynchronize(I->stream), "tl_set_tip_states_all");
}

int tl_launch_count(const tl_instance* inst, unsigned long long* out) {
    if (!inst || !out) return TL_ERR_ARG;
    *out = reinterpret_cast<const Instance*>(inst)->launches;
    return TL_OK;
}

int tl_set_tip_partials(tl_instance* inst, int tip, const double* partials) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (tip < 0 || tip >= I->n_tips) return fail(I, TL_ERR_INDEX, "tip %d out of range", tip);
    if (!partials) return fail(I, TL_ERR_ARG, "partials is null");
    for (size_t i = 0; i < (size_t)I->P * I->S; ++i)
        if (!std::isfinite(partials[i]) || partials[i] < 0)
            return fail(I, TL_ERR_NUMERIC, "tip partial %zu is negative or not finite", i);
    const size_t n = (size_t)I->R * I->Ppad * I->Spad;
    int rc;
    if (I->prec == kTF32) {
        // tensor-core instances keep tip partials in one pool the TMA map covers
        if (!I->tc_tip_pool) {
            if ((rc = dev_alloc(I, &I->tc_tip_pool, n * sizeof(float) * I->n_tips, "tip partials")))
                return rc;
            if ((rc = tc_set_tip_pool(I))) return rc;
        }
        I->tip_part[tip] = I->tc_tip_pool + n * tip;
    } else if (!I->tip_part[tip]) {
        if ((rc = dev_alloc(I, &I->tip_part[tip], n * I->elt, "tip partials"))) return rc;
    }
    std::vector<char> h(n * I->elt);
    for (int r = 0; r < I->R; ++r)
        for (int p = 0; p < I->Ppad; ++p)
            for (int s = 0; s < I->Spad; ++s) {
                double v = (s >= I->S) ? 0.0 : (p < I->P ? partials[(size_t)p * I->S + s] : 1.0);
                size_t off = ((size_t)r * I->Ppad + p) * I->Spad + s;
                if (I->elt == 8) reinterpret_cast<double*>(h.data())[off] = v;
                else if (I->prec == kTF32)
                    reinterpret_cast<float*>(h.data())[off] =
                        I->split_partials ? (float)v : tf32_host((float)v);
                else reinterpret_cast<float*>(h.data())[off] = (float)v;
            }
    cudaMemcpyAsync(I->tip_part[tip], h.data(), h.size(), cudaMemcpyHostToDevice, I->stream);
    I->h_buf[tip] = I->tip_part[tip];
    I->h_tipst[tip] = nullptr;
    if ((rc = h2d(I, I->d_tipst + tip, &I->h_tipst[tip], sizeof(int8_t*)))) return rc;
    if ((rc = h2d(I, I->d_buf + tip, &I->h_buf[tip], sizeof(void*)))) return rc;
    I->tip_set[tip] = 2;
    return cuda_check(I, cudaStreamSynchronize(I->stream), "tl_set_tip_partials");
}

int tl_set_pattern_weights(tl_instance* inst, const double* w) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (!w) return fail(I, TL_ERR_ARG, "weights is null");
    std::vector<double> h(I->Ppad, 0.0);
    for (int p = 0; p < I->P; ++p) {
        if (!std::isfinite(w[p]) || w[p] < 0)
            return fail(I, TL_ERR_NUMERIC, "pattern weight %d is negative or not finite", p);
        h[p] = w[p];
    }
    return h2d(I, I->d_patw, h.data(), sizeof(double) * I->Ppad);
}

int tl_set_category_rates(tl_instance* inst, const double* rates) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (!rates) return fail(I, TL_ERR_ARG, "rates is null");
    for (int r = 0; r < I->R; ++r)
        if (!std::isfinite(rates[r]) || rates[r] < 0)
            return fail(I, TL_ERR_NUMERIC, "category rate %d is negative or not finite", r);
    for (int r = 0; r < I->R; ++r) I->h_rates[r] = rates[r];
    return TL_OK;
}

int tl_set_category_weights(tl_instance* inst, const double* w) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (!w) return fail(I, TL_ERR_ARG, "weights is null");
    for (int r = 0; r < I->R; ++r)
        if (!std::isfinite(w[r]) || w[r] < 0)
            return fail(I, TL_ERR_NUMERIC, "category weight %d is negative or not finite", r);
    for (int r = 0; r < I->R; ++r) I->h_catw[r] = w[r];
    return TL_OK;
}

static int stage(Instance* I, const double* a, int na, const double* b, int nb) {
    if ((size_t)(na + nb) > I->tmp_cap) return fail(I, TL_ERR_ARG, "staging too large");
    std::vector<double> h((size_t)na + nb);
    if (na) std::memcpy(h.data(), a, sizeof(double) * na);
    if (nb) std::memcpy(h.data() + na, b, sizeof(double) * nb);
    return h2d(I, I->d_tmp, h.data(), sizeof(double) * h.size());
}

static int set_model(tl_instance* inst, int model, int kind, const double* params, int n_params,
                     const double* freqs, int n_freqs, bool check) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (model < 0 || model >= I->n_models) return fail(I, TL_ERR_INDEX, "model %d out of range", model);
    int want_p = 0, want_f = 0;
    switch (kind) {
        case TL_MODEL_HKY: want_p = 1; want_f = 4; break;
        case TL_MODEL_GTR: want_p = 6; want_f = 4; break;
        case TL_MODEL_GY94: want_p = 2; want_f = 12; break;
        case TL_MODEL_REV: want_p = I->S * I->S; want_f = I->S; break;
        case TL_MODEL_GY94RE: want_p = 2 + TL_GY94_PAIRS; want_f = 12; break;
        default: return fail(I, TL_ERR_ARG, "unknown model kind %d", kind);
    }
    if ((kind == TL_MODEL_HKY || kind == TL_MODEL_GTR) && I->S != 4)
        return fail(I, TL_ERR_ARG, "nucleotide model on a %d-state instance", I->S);
    if ((kind == TL_MODEL_GY94 || kind == TL_MODEL_GY94RE) && I->S != 61)
        return fail(I, TL_ERR_ARG, "GY94 needs 61 states, instance has %d", I->S);
    if (n_params != want_p || n_freqs != want_f || !params || !freqs)
        return fail(I, TL_ERR_ARG, "model kind %d takes %d params and %d freqs", kind, want_p, want_f);
    for (int i = 0; i < n_params; ++i)  // random effects (after kappa, omega) may be negative
        if (!std::isfinite(params[i]) || (params[i] < 0 && !(kind == TL_MODEL_GY94RE && i >= 2)))
            return fail(I, TL_ERR_NUMERIC, "parameter %d is negative or not finite", i);
    for (int i = 0; i < n_freqs; ++i)
        if (!std::isfinite(freqs[i]) || freqs[i] <= 0)
            return fail(I, TL_ERR_NUMERIC, "frequency %d is not positive and finite", i);
    if (n_params + n_freqs > (int)I->tmp_cap) {
        dev_free(I, I->d_tmp);
        I->tmp_cap = n_params + n_freqs + 1024;
        int rc = dev_alloc(I, &I->d_tmp, sizeof(double) * I->tmp_cap, "staging");
        if (rc) return rc;
    }
    int rc = stage(I, params, n_params, freqs, n_freqs);
    if (rc) return rc;
    I->models[model].ready = false;
    I->models[model].kind = kind;
    I->models[model].n_params = n_params;
    return launch_build_model(I, model, kind, I->d_tmp, n_params, I->d_tmp + n_params, n_freqs,
                              check);
}

int tl_set_model(tl_instance* inst, int model, int kind, const double* params, int n_params,
                 const double* freqs, int n_freqs) {
    return set_model(inst, model, kind, params, n_params, freqs, n_freqs, true);
}

int tl_set_model_async(tl_instance* inst, int model, int kind, const double* params, int n_params,
                       const double* freqs, int n_freqs) {
    return set_model(inst, model, kind, params, n_params, freqs, n_freqs, false);
}

int tl_set_rate_matrix(tl_instance* inst, int model, const double* Q, const double* pi) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (model < 0 || model >= I->n_models) return fail(I, TL_ERR_INDEX, "model %d out of range", model);
    if (!Q || !pi) return fail(I, TL_ERR_ARG, "null input");
    const int S = I->S, Sp = I->Spad;
    std::vector<double> q((size_t)Sp * Sp, 0.0), p(Sp, 0.0);
    for (int i = 0; i < S; ++i) {
        if (!(pi[i] > 0) || !std::isfinite(pi[i])) return fail(I, TL_ERR_NUMERIC, "pi[%d] not positive", i);
        p[i] = pi[i];
        for (int j = 0; j < S; ++j) {
            if (!std::isfinite(Q[i * S + j])) return fail(I, TL_ERR_NUMERIC, "Q not finite");
            q[(size_t)i * Sp + j] = Q[i * S + j];
        }
    }
    ModelDev& M = I->models[model];
    cudaMemcpyAsync(M.Q, q.data(), sizeof(double) * q.size(), cudaMemcpyHostToDevice, I->stream);
    cudaMemcpyAsync(M.pi, p.data(), sizeof(double) * Sp, cudaMemcpyHostToDevice, I->stream);
    M.n_dq = 0;
    M.kind = 0;
    M.n_params = 0;
    M.ready = false;
    return launch_eigen_from_q(I, model, true);
}

int tl_set_eigen(tl_instance* inst, int model, const double* V, const double* Vinv,
                 const double* lambda, const double* pi) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (model < 0 || model >= I->n_models) return fail(I, TL_ERR_INDEX, "model %d out of range", model);
    if (!V || !Vinv || !lambda || !pi) return fail(I, TL_ERR_ARG, "null input");
    const int S = I->S, Sp = I->Spad;
    std::vector<double> v((size_t)Sp * Sp, 0.0), vi((size_t)Sp * Sp, 0.0), l(Sp, 0.0), p(Sp, 0.0);
    for (int i = 0; i < S; ++i) {
        l[i] = lambda[i];
        p[i] = pi[i];
        for (int j = 0; j < S; ++j) {
            v[(size_t)i * Sp + j] = V[i * S + j];
            vi[(size_t)i * Sp + j] = Vinv[i * S + j];
        }
    }
    for (double x : v) if (!std::isfinite(x)) return fail(I, TL_ERR_NUMERIC, "V not finite");
    for (double x : vi) if (!std::isfinite(x)) return fail(I, TL_ERR_NUMERIC, "Vinv not finite");
    ModelDev& M = I->models[model];
    cudaMemcpyAsync(M.V, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, I->stream);
    cudaMemcpyAsync(M.Vinv, vi.data(), sizeof(double) * vi.size(), cudaMemcpyHostToDevice, I->stream);
    cudaMemcpyAsync(M.lam, l.data(), sizeof(double) * Sp, cudaMemcpyHostToDevice, I->stream);
    cudaMemcpyAsync(M.pi, p.data(), sizeof(double) * Sp, cudaMemcpyHostToDevice, I->stream);
    M.n_dq = 0;
    M.kind = 0;
    M.n_params = 0;
    int rc = launch_q_from_eigen(I, model);
    if (rc) return rc;
    return launch_model_working_copies(I, model);
}

int tl_get_model(tl_instance* inst, int model, double* Q, double* pi, double* dq, int* n_dq) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (model < 0 || model >= I->n_models) return fail(I, TL_ERR_INDEX, "model %d out of range", model);
    ModelDev& M = I->models[model];
    if (!M.ready) return fail(I, TL_ERR_STATE, "model %d not set", model);
    const int S = I->S, Sp = I->Spad;
    std::vector<double> q((size_t)Sp * Sp), p(Sp), d((size_t)kMaxDq * Sp * Sp);
    cudaMemcpyAsync(q.data(), M.Q, sizeof(double) * q.size(), cudaMemcpyDeviceToHost, I->stream);
    cudaMemcpyAsync(p.data(), M.pi, sizeof(double) * Sp, cudaMemcpyDeviceToHost, I->stream);
    cudaMemcpyAsync(d.data(), M.dQ, sizeof(double) * d.size(), cudaMemcpyDeviceToHost, I->stream);
    int rc = cuda_check(I, cudaStreamSynchronize(I->stream), "tl_get_model");
    if (rc) return rc;
    for (int i = 0; i < S; ++i) {
        if (pi) pi[i] = p[i];
        for (int j = 0; j < S; ++j)
            if (Q) Q[i * S + j] = q[(size_t)i * Sp + j];
    }
    if (dq)
        for (int k = 0; k < M.n_dq; ++k)
            for (int i = 0; i < S; ++i)
                for (int j = 0; j < S; ++j)
                    dq[((size_t)k * S + i) * S + j] = d[((size_t)k * Sp + i) * Sp + j];
    if (n_dq) *n_dq = M.n_dq;
    return TL_OK;
}

int tl_update_matrices(tl_instance* inst, int model, const int* p_idx, const int* dp_idx,
                       const double* edge_len, int count) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (model < 0 || model >= I->n_models) return fail(I, TL_ERR_INDEX, "model %d out of range", model);
    if (!I->models[model].ready) return fail(I, TL_ERR_STATE, "model %d not set", model);
    if (count < 0 || (count > 0 && (!p_idx || !edge_len))) return fail(I, TL_ERR_ARG, "bad arguments");
    for (int i = 0; i < count; ++i) {
        if (p_idx[i] < 0 || p_idx[i] >= I->n_mats)
            return fail(I, TL_ERR_INDEX, "p_idx[%d]=%d out of range", i, p_idx[i]);
        if (dp_idx && (dp_idx[i] < -1 || dp_idx[i] >= I->n_mats))
            return fail(I, TL_ERR_INDEX, "dp_idx[%d]=%d out of range", i, dp_idx[i]);
        if (!std::isfinite(edge_len[i]) || edge_len[i] < 0)
            return fail(I, TL_ERR_NUMERIC, "edge_len[%d] is negative or not finite", i);
    }
    // staging: rates [R] | lengths [count] in d_tmp; indices in d_ops area 3
    if ((size_t)(I->R + count) > I->tmp_cap) {
        dev_free(I, I->d_tmp);
        I->tmp_cap = I->R + count + 1024;
        int rc = dev_alloc(I, &I->d_tmp, sizeof(double) * I->tmp_cap, "staging");
        if (rc) return rc;
    }
    int rc = stage(I, I->h_rates, I->R, edge_len, count);
    if (rc) return rc;
    std::vector<int> idx(2 * (size_t)count);
    for (int i = 0; i < count; ++i) {
        idx[i] = p_idx[i];
        idx[count + i] = dp_idx ? dp_idx[i] : -1;
    }
    void* d_idx = nullptr;
    Extra& X = extra(I);
    if ((rc = upload(I, X.areas[3], idx.data(), sizeof(int) * idx.size(), &d_idx))) return rc;
    rc = launch_update_matrices(I, model, (const int*)d_idx, (const int*)d_idx + count,
                                I->d_tmp + I->R, count);
    if (rc) return rc;
    for (int i = 0; i < count; ++i) {
        I->mat_set[p_idx[i]] = 1;
        I->mat_len[p_idx[i]] = edge_len[i];
        I->mat_model[p_idx[i]] = model;
    }
    for (int i = 0; i < count; ++i)
        if (dp_idx && dp_idx[i] >= 0) {
            I->mat_set[dp_idx[i]] = 1;
            I->mat_model[dp_idx[i]] = -1;
        }
    return TL_OK;
}

int tl_get_matrix(tl_instance* inst, int mat, double* out) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (mat < 0 || mat >= I->n_mats) return fail(I, TL_ERR_INDEX, "matrix %d out of range", mat);
    if (!out) return fail(I, TL_ERR_ARG, "out is null");
    const int S = I->S, Sp = I->Spad;
    std::vector<double> h((size_t)I->R * Sp * Sp);
    cudaMemcpyAsync(h.data(), I->d_mat64 + (size_t)mat * I->R * Sp * Sp, sizeof(double) * h.size(),
                    cudaMemcpyDeviceToHost, I->stream);
    int rc = cuda_check(I, cudaStreamSynchronize(I->stream), "tl_get_matrix");
    if (rc) return rc;
    for (int r = 0; r < I->R; ++r)
        for (int i = 0; i < S; ++i)
            for (int j = 0; j < S; ++j)
                out[((size_t)r * S + i) * S + j] = h[((size_t)r * Sp + i) * Sp + j];
    return TL_OK;
}

extern "C++" {
template <typename T>
static void adj_fill(const Instance* I, const tl_adj_op& o, const double* P0, const double* P1,
                     const int row[2], std::vector<char>& table, size_t at) {
    AdjOp<T> d;
    std::memset(&d, 0, sizeof d);
    d.q = o.parent_pre >= 0 ? reinterpret_cast<const T*>(I->h_buf[o.parent_pre]) : nullptr;
    d.pn = reinterpret_cast<const T*>(I->h_buf[o.parent_post]);
    d.en = I->h_scale[o.parent_post];
    for (int c = 0; c < 2; ++c) {
        const int v = o.child[c];
        if (v < I->n_tips && I->tip_set[v] == 1) {
            d.st[c] = I->h_tipst[v];
        } else {
            d.part[c] = reinterpret_cast<const T*>(I->h_buf[v]);
            d.ec[c] = v < I->n_tips ? nullptr : I->h_scale[v];
        }
        d.row[c] = row[c];
    }
    d.P[0] = P0;
    d.P[1] = P1;
    std::memcpy(table.data() + at * sizeof d, &d, sizeof d);
}
}  // extern "C++"

int tl_adjoint(tl_instance* inst, const tl_adj_op* ops, int count, int model, unsigned flags,
               double* out_grad, int n_grad, double* out_dQ, double* out_dtheta, int n_theta) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    if (model < 0 || model >= I->n_models || !I->models[model].ready)
        return fail(I, TL_ERR_STATE, "model %d not set", model);
    if (count < 0 || (count > 0 && !ops)) return fail(I, TL_ERR_ARG, "bad op list");
    if (n_grad < 0 || (n_grad > 0 && !out_grad)) return fail(I, TL_ERR_ARG, "bad out_grad");
    if (flags & ~TL_ADJ_FIRST_ORDER) return fail(I, TL_ERR_ARG, "unknown flags 0x%x", flags);
    const ModelDev& Mo = I->models[model];
    if (out_dtheta && n_theta != Mo.n_params)
        return fail(I, TL_ERR_ARG, "model %d has %d parameters, n_theta is %d", model, Mo.n_params,
                    n_theta);
    const int NB = I->n_bufs, SS = I->Spad * I->Spad;
    const size_t mat_doubles = (size_t)I->R * SS;
    const size_t op_bytes = I->elt == 8 ? sizeof(AdjOp<double>) : sizeof(AdjOp<float>);
    std::vector<char> table(op_bytes * std::max(count, 1));
    std::vector<AdjEdge> edges;
    std::vector<int> edge_id, seen(std::max(n_grad, 1), 0);
    for (int k = 0; k < count; ++k) {
        const tl_adj_op& o = ops[k];
        if (o.parent_post < I->n_tips || o.parent_post >= NB ||
            !I->buf_written[o.parent_post - I->n_tips])
            return fail(I, TL_ERR_STATE, "adjoint op %d: parent_post %d holds no post-order partial",
                        k, o.parent_post);
        if (o.parent_pre != -1 && (o.parent_pre < I->n_tips || o.parent_pre >= NB ||
                                   !I->buf_written[o.parent_pre - I->n_tips]))
            return fail(I, TL_ERR_STATE, "adjoint op %d: parent_pre %d holds no pre-order partial",
                        k, o.parent_pre);
        const double* P[2];
        int row[2];
        for (int c = 0; c < 2; ++c) {
            const int v = o.child[c], m = o.mat[c];
            if (v < 0 || v >= NB) return fail(I, TL_ERR_INDEX, "adjoint op %d: child %d", k, v);
            if (v < I->n_tips ? !I->tip_set[v] : !I->buf_written[v - I->n_tips])
                return fail(I, TL_ERR_STATE, "adjoint op %d: child %d holds no data", k, v);
            if (m < 0 || m >= I->n_mats) return fail(I, TL_ERR_INDEX, "adjoint op %d: matrix %d", k, m);
            if (!I->mat_set[m] || I->mat_model[m] != model)
                return fail(I, TL_ERR_STATE, "adjoint op %d: matrix %d is not a transition matrix "
                            "of model %d", k, m, model);
            P[c] = I->d_mat64 + (size_t)m * mat_doubles;
            row[c] = -1;
            const int e = o.edge[c];
            if (e >= 0) {
                if (e >= n_grad) return fail(I, TL_ERR_INDEX, "adjoint op %d: edge %d >= n_grad", k, e);
                if (seen[e]) return fail(I, TL_ERR_ORDER, "adjoint op %d: edge %d listed twice", k, e);
                seen[e] = 1;
                row[c] = (int)edges.size();
                edges.push_back({P[c], I->mat_len[m]});
                edge_id.push_back(e);
            }
        }
        if (I->elt == 8) adj_fill<double>(I, o, P[0], P[1], row, table, k);
        else adj_fill<float>(I, o, P[0], P[1], row, table, k);
    }
    const int E = (int)edges.size();
    int rc;
    if ((size_t)I->R > I->tmp_cap) {
        dev_free(I, I->d_tmp);
        I->tmp_cap = I->R + 1024;
        if ((rc = dev_alloc(I, &I->d_tmp, sizeof(double) * I->tmp_cap, "staging"))) return rc;
    }
    if ((rc = stage(I, I->h_rates, I->R, nullptr, 0))) return rc;
    // scratch: [coef | mpart | M | gpart | G | grad | dQ | theta]
    const int n_chunks = adj_chunks(I, std::max(count, 1));
    const bool nuc = use_nuc(I);
    const size_t n_coef = nuc ? 0 : (size_t)count * I->Ppad;
    const size_t n_mpart = (size_t)E * mat_doubles * n_chunks;
    const size_t n_M = (size_t)E * mat_doubles;
    const size_t n_gpart = (size_t)SS * std::max(E, 1);
    const size_t n_theta_dev = std::max<size_t>(2 + TL_GY94_PAIRS + kMaxDq, SS);
    if ((rc = ensure_scratch(I, n_coef + n_mpart + n_M + n_gpart + SS + E + SS + n_theta_dev)))
        return rc;
    double* d_coef = I->d_red;
    double* d_mpart = d_coef + n_coef;
    double* d_M = d_mpart + n_mpart;
    double* d_gpart = d_M + n_M;
    double* d_G = d_gpart + n_gpart;
    double* d_grad = d_G + SS;
    double* d_dQ = d_grad + E;
    double* d_theta = d_dQ + SS;
    void* d_ops = area(I, 1, table.size() + sizeof(AdjEdge) * std::max(E, 1) + 16, &rc);
    if (rc) return rc;
    AdjEdge* d_edges = reinterpret_cast<AdjEdge*>((char*)d_ops + ((table.size() + 15) / 16) * 16);
    if ((rc = h2d(I, d_ops, table.data(), table.size()))) return rc;
    if (E > 0 && (rc = h2d(I, d_edges, edges.data(), sizeof(AdjEdge) * E))) return rc;
    if (count > 0 && E > 0) {
        if ((rc = launch_adj_accumulate(I, d_ops, count, n_chunks, n_M, d_coef, d_mpart, model)))
            return rc;
        if ((rc = launch_adj_sum_chunks(I, d_mpart, n_M, n_chunks, d_M))) return rc;
        const bool first = flags & TL_ADJ_FIRST_ORDER;
        if ((rc = launch_adj_finish(I, model, d_M, d_edges, E, first, d_gpart, d_grad))) return rc;
        if ((rc = reduce_fixed(I, d_gpart, SS, E, d_G))) return rc;
    } else {
        cudaMemsetAsync(d_G, 0, sizeof(double) * SS, I->stream);
    }
    if ((rc = launch_adj_params(I, model, d_G, flags & TL_ADJ_FIRST_ORDER, d_dQ, d_theta)))
        return rc;
    std::vector<double> h_grad(std::max(E, 1)), h_dQ(SS), h_theta(n_theta_dev);
    if (E > 0) cudaMemcpyAsync(h_grad.data(), d_grad, sizeof(double) * E, cudaMemcpyDeviceToHost, I->stream);
    cudaMemcpyAsync(h_dQ.data(), d_dQ, sizeof(double) * SS, cudaMemcpyDeviceToHost, I->stream);
    cudaMemcpyAsync(h_theta.data(), d_theta, sizeof(double) * n_theta_dev, cudaMemcpyDeviceToHost,
                    I->stream);
    if ((rc = cuda_check(I, cudaStreamSynchronize(I->stream), "tl_adjoint"))) return rc;
    if ((rc = check_numeric_flag(I))) return rc;
    if (out_grad) {
        for (int i = 0; i < n_grad; ++i) out_grad[i] = 0.0;
        for (int e = 0; e < E; ++e) out_grad[edge_id[e]] = h_grad[e];
    }
    if (out_dQ)
        for (int i = 0; i < I->S; ++i)
            for (int j = 0; j < I->S; ++j) out_dQ[i * I->S + j] = h_dQ[(size_t)i * I->Spad + j];
    if (out_dtheta)
        for (int k = 0; k < n_theta; ++k) out_dtheta[k] = h_theta[k];
    return TL_OK;
}

int tl_ratio_heights(int n_tips, const int* parent, const double* tip_height, const double* ratio,
                     double root_height, const double* rate, double* out_height,
                     double* out_len, void* stream) {
    return ratio_run(n_tips, parent, tip_height, ratio, root_height, rate, nullptr, out_height,
                     out_len, nullptr, nullptr, nullptr, stream, &g_create_err);
}

int tl_ratio_gradient(int n_tips, const int* parent, const double* tip_height, const double* ratio,
                      double root_height, const double* rate, const double* grad_len,
                      double* out_grad_ratio, double* out_grad_root_height,
                      double* out_grad_rate, void* stream) {
    if (!grad_len) {
        g_create_err = "grad_len is null";
        return TL_ERR_ARG;
    }
    return ratio_run(n_tips, parent, tip_height, ratio, root_height, rate, grad_len, nullptr,
                     nullptr, out_grad_ratio, out_grad_root_height, out_grad_rate, stream,
                     &g_create_err);
}

int tl_get_partials(tl_instance* inst, int buf, double* out, int32_t* exponents) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (buf < 0 || buf >= I->n_bufs) return fail(I, TL_ERR_INDEX, "buffer %d out of range", buf);
    if (!out) return fail(I, TL_ERR_ARG, "out is null");
    if (!I->h_buf[buf]) return fail(I, TL_ERR_STATE, "buffer %d holds tip states, not partials", buf);
    const size_t n = (size_t)I->R * I->Ppad * I->Spad;
    std::vector<char> h(n * I->elt);
    std::vector<int> e(I->Ppad, 0);
    cudaMemcpyAsync(h.data(), I->h_buf[buf], h.size(), cudaMemcpyDeviceToHost, I->stream);
    if (I->h_scale[buf])
        cudaMemcpyAsync(e.data(), I->h_scale[buf], sizeof(int) * I->Ppad, cudaMemcpyDeviceToHost, I->stream);
    int rc = cuda_check(I, cudaStreamSynchronize(I->stream), "tl_get_partials");
    if (rc) return rc;
    for (int r = 0; r < I->R; ++r)
        for (int p = 0; p < I->P; ++p)
            for (int s = 0; s < I->S; ++s) {
                size_t src = ((size_t)r * I->Ppad + p) * I->Spad + s;
                out[((size_t)r * I->P + p) * I->S + s] =
                    I->elt == 8 ? reinterpret_cast<double*>(h.data())[src]
                                : (double)reinterpret_cast<float*>(h.data())[src];
            }
    if (exponents)
        for (int p = 0; p < I->P; ++p) exponents[p] = e[p];
    return TL_OK;
}

int tl_update_partials(tl_instance* inst, const tl_op* ops, int count) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    if (count < 0 || (count > 0 && !ops)) return fail(I, TL_ERR_ARG, "bad op list");
    if (count == 0) return TL_OK;
    int rc;
    if (use_tc(I)) {
        // depth-first order (the planner's): each op's child produced by
        // the op just before is marked, and the fused kernel keeps it on chip
        const bool fused = tc_fused_enabled(I) != 0;
        PostPlan plan;
        if ((rc = plan_post(I, ops, count, &plan, !fused))) return rc;
        const size_t bytes = (size_t)count * kTcOpBytes;
        void* d = area(I, 0, bytes, &rc);
        if (rc) return rc;
        if (fused) rc = launch_post_tc_fused(I, plan.dev.data(), count, d, bytes);
        else rc = launch_post_tc(I, ops, count, d, bytes);
        if (rc) return rc;
    } else if (use_nuc(I)) {
        PostPlan plan;
        if ((rc = plan_post(I, ops, count, &plan, false))) return rc;
        void* d_ops = nullptr;
        if ((rc = upload(I, extra(I).areas[0], plan.dev.data(), sizeof(DevPostOp) * count, &d_ops)))
            return rc;
        if ((rc = launch_post4(I, (const DevPostOp*)d_ops, count, plan.n_slots))) return rc;
    } else {
        PostPlan plan;
        if ((rc = plan_post(I, ops, count, &plan, true))) return rc;
        if ((rc = launch_post_generic(I, ops, count))) return rc;
    }
    for (int k = 0; k < count; ++k) I->buf_written[ops[k].dest - I->n_tips] = 1;
    return TL_OK;
}

int tl_update_partials_eigen(tl_instance* inst, int model, const tl_eig_op* ops, int count) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (I->prec != kF64) return fail(I, TL_ERR_UNSUPPORTED, "on-the-fly matrices need TL_PREC_F64");
    if (model < 0 || model >= I->n_models || !I->models[model].ready)
        return fail(I, TL_ERR_STATE, "model %d not set", model);
    if (count < 0 || (count > 0 && !ops)) return fail(I, TL_ERR_ARG, "bad op list");
    if (count == 0) return TL_OK;
    const int NB = I->n_bufs;
    std::vector<int> prod(NB, -1), level(count, 0);
    for (int k = 0; k < count; ++k) {
        const int d = ops[k].dest;
        if (d < I->n_tips || d >= NB) return fail(I, TL_ERR_INDEX, "op %d: dest %d", k, d);
        if (prod[d] >= 0) return fail(I, TL_ERR_ORDER, "op %d: buffer %d written twice", k, d);
        prod[d] = k;
    }
    for (int k = 0; k < count; ++k) {
        const tl_eig_op& o = ops[k];
        const int ch[2] = {o.child1, o.child2};
        const double len[2] = {o.len1, o.len2};
        for (int c = 0; c < 2; ++c) {
            const int v = ch[c];
            if (v < 0 || v >= NB) return fail(I, TL_ERR_INDEX, "op %d: child %d", k, v);
            if (!std::isfinite(len[c]) || len[c] < 0)
                return fail(I, TL_ERR_NUMERIC, "op %d: edge length not finite and >= 0", k);
            if (v < I->n_tips) {
                if (!I->tip_set[v]) return fail(I, TL_ERR_STATE, "op %d: tip %d not set", k, v);
            } else if (prod[v] >= 0) {
                if (prod[v] >= k)
                    return fail(I, TL_ERR_ORDER, "op %d reads buffer %d before it is written", k, v);
                level[k] = std::max(level[k], level[prod[v]] + 1);
            } else if (!I->buf_written[v - I->n_tips]) {
                return fail(I, TL_ERR_STATE, "op %d: child %d holds no data", k, v);
            }
        }
    }
    const int n_levels = *std::max_element(level.begin(), level.end()) + 1;
    std::vector<int> start(n_levels + 1, 0);
    for (int k = 0; k < count; ++k) start[level[k] + 1]++;
    for (int L = 0; L < n_levels; ++L) start[L + 1] += start[L];
    std::vector<EigOp> dev(count);
    {
        std::vector<int> fill(start.begin(), start.end() - 1);
        for (int k = 0; k < count; ++k) {
            EigOp e;
            e.dest = ops[k].dest;
            e.child[0] = ops[k].child1;
            e.child[1] = ops[k].child2;
            e.pad = 0;
            e.len[0] = ops[k].len1;
            e.len[1] = ops[k].len2;
            dev[fill[level[k]]++] = e;
        }
    }
    int rc;
    if ((size_t)I->R > I->tmp_cap) {
        dev_free(I, I->d_tmp);
        I->tmp_cap = I->R + 1024;
        if ((rc = dev_alloc(I, &I->d_tmp, sizeof(double) * I->tmp_cap, "staging"))) return rc;
    }
    void* d_ops = area(I, 0, sizeof(EigOp) * count, &rc);
    if (rc) return rc;
    if ((rc = h2d(I, d_ops, dev.data(), sizeof(EigOp) * count))) return rc;
    if ((rc = launch_post_eig(I, model, reinterpret_cast<const EigOp*>(d_ops), start.data(),
                              n_levels)))
        return rc;
    for (int k = 0; k < count; ++k) I->buf_written[ops[k].dest - I->n_tips] = 1;
    return TL_OK;
}

static int root_common(Instance* I, int root, int model, double* d_site, double* d_out) {
    if (root < 0 || root >= I->n_bufs) return fail(I, TL_ERR_INDEX, "root %d out of range", root);
    if (root >= I->n_tips ? !I->buf_written[root - I->n_tips] : !I->tip_set[root])
        return fail(I, TL_ERR_STATE, "root buffer %d holds no data", root);
    if (model < 0 || model >= I->n_models || !I->models[model].ready)
        return fail(I, TL_ERR_STATE, "model %d not set", model);
    int rc;
    if (use_tc(I)) {
        if (root < I->n_tips) return fail(I, TL_ERR_UNSUPPORTED, "root must be an internal buffer");
        const int parts = I->Ppad / 128;
        if ((rc = ensure_scratch(I, parts))) return rc;
        if ((rc = h2d(I, I->d_tmp, I->h_catw, sizeof(double) * I->R))) return rc;
        if ((rc = launch_root_tc(I, root - I->n_tips, model, d_site, I->d_red, parts))) return rc;
        return reduce_fixed(I, I->d_red, 1, parts, d_out);
    }
    if (use_nuc(I)) {
        const int n_tiles = nuc_tiles(I);
        if ((rc = ensure_scratch(I, n_tiles))) return rc;
        int kind = kInternal, idx = root - I->n_tips;
        if (root < I->n_tips) {
            kind = I->tip_set[root] == 1 ? kTipStates : kTipPartials;
            idx = root;
        }
        if ((rc = launch_root4(I, kind, idx, model, d_site, I->d_red))) return rc;
        return reduce_fixed(I, I->d_red, 1, n_tiles, d_out);
    }
    const int parts = (I->Ppad + 127) / 128;
    if ((rc = ensure_scratch(I, parts))) return rc;
    if ((rc = launch_root_generic(I, root, model, d_site, I->d_red, parts))) return rc;
    return reduce_fixed(I, I->d_red, 1, parts, d_out);
}

int tl_root_loglik(tl_instance* inst, int root, int model, double* out_logl, double* out_site) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    if (!out_logl) return fail(I, TL_ERR_ARG, "out_logl is null");
    int rc;
    if ((rc = ensure_out(I, 1 + (size_t)I->Ppad))) return rc;
    double* d_out = extra(I).d_out;
    double* d_site = out_site ? d_out + 1 : nullptr;
    if ((rc = root_common(I, root, model, d_site, d_out))) return rc;
    cudaMemcpyAsync(out_logl, d_out, sizeof(double), cudaMemcpyDeviceToHost, I->stream);
    if (out_site)
        cudaMemcpyAsync(out_site, d_site, sizeof(double) * I->P, cudaMemcpyDeviceToHost, I->stream);
    if ((rc = cuda_check(I, cudaStreamSynchronize(I->stream), "tl_root_loglik"))) return rc;
    return check_numeric_flag(I);
}

int tl_root_loglik_dev(tl_instance* inst, int root, int model, double* out_logl_dev) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    if (!out_logl_dev) return fail(I, TL_ERR_ARG, "out is null");
    return root_common(I, root, model, nullptr, out_logl_dev);
}

static int pre_common(Instance* I, const tl_pre_op* ops, int count, int model, int n_grad,
                      bool store_all, double* d_grad_out, int dgen = 0) {
    if (count < 0 || (count > 0 && !ops)) return fail(I, TL_ERR_ARG, "bad op list");
    if (model < 0 || model >= I->n_models || !I->models[model].ready)
        return fail(I, TL_ERR_STATE, "model %d not set", model);
    if (n_grad < 0) return fail(I, TL_ERR_ARG, "n_grad < 0");
    PrePlan plan;
    int rc = plan_pre(I, ops, count, n_grad, store_all, &plan);
    if (rc) return rc;
    const int E = (int)plan.edge_map.size();
    if (use_tc(I)) {
        const int n_tiles = I->Ppad / 128;
        if ((rc = ensure_scratch(I, (size_t)std::max(E, 1) * n_tiles))) return rc;
        std::vector<int> row(std::max(n_grad, 1), -1);
        for (int k = 0; k < E; ++k) row[plan.edge_map[k]] = k;
        const size_t bytes = (size_t)count * 3 * kTcOpBytes;
        void* d = area(I, 1, bytes, &rc);
        if (rc) return rc;
        if ((rc = launch_pre_tc(I, ops, count, row.data(), model, I->d_red, d, bytes, dgen)))
            return rc;
        if ((rc = ensure_out(I, (size_t)E))) return rc;
        if ((rc = reduce_fixed(I, I->d_red, E, n_tiles, extra(I).d_out))) return rc;
    } else if (use_nuc(I)) {
        const int n_tiles = nuc_tiles_pre(I);
        if ((rc = ensure_scratch(I, (size_t)std::max(E, 1) * n_tiles))) return rc;
        void* d_ops = nullptr;
        if ((rc = upload(I, extra(I).areas[1], plan.dev.data(), sizeof(DevPreOp) * count, &d_ops)))
            return rc;
        if ((rc = launch_pre4(I, (const DevPreOp*)d_ops, count, plan.n_slots, model, I->d_red,
                              dgen)))
            return rc;
        if ((rc = ensure_out(I, (size_t)E))) return rc;
        if ((rc = reduce_fixed(I, I->d_red, E, n_tiles, extra(I).d_out))) return rc;
    } else {
        // generic path: q partials always go through buffers; ops whose q
        // output is consumed but unnamed are rejected by plan_pre (pre >= 0
        // is required to name a consumed q).
        const int parts = generic_parts(I);
        if ((rc = ensure_scratch(I, (size_t)std::max(E, 1) * parts))) return rc;
        std::vector<tl_pre_op> g(ops, ops + count);
        std::vector<int> row(std::max(n_grad, 1), -1);
        for (int k = 0; k < E; ++k) row[plan.edge_map[k]] = k;
        for (auto& o : g)
            for (int c = 0; c < 2; ++c) o.edge[c] = o.edge[c] >= 0 ? row[o.edge[c]] : -1;
        if ((rc = launch_pre_generic(I, g.data(), count, model, I->d_red, parts))) return rc;
        if ((rc = ensure_out(I, (size_t)E))) return rc;
        if ((rc = reduce_fixed(I, I->d_red, E, parts, extra(I).d_out))) return rc;
    }
    if (use_nuc(I)) {
        for (int b : plan.stored) I->buf_written[b - I->n_tips] = 1;
    } else {
        for (int k = 0; k < count; ++k)
            for (int c = 0; c < 2; ++c)
                if (ops[k].pre[c] >= 0) I->buf_written[ops[k].pre[c] - I->n_tips] = 1;
    }
    if (d_grad_out && n_grad > 0) {
        void* d_map = nullptr;
        if (E > 0 && (rc = upload(I, extra(I).areas[4], plan.edge_map.data(), sizeof(int) * E, &d_map)))
            return rc;
        k_scatter<<<1, 256, 0, I->stream>>>(extra(I).d_out, (const int*)d_map, E, d_grad_out, n_grad);
        I->launches += 1;
        if ((rc = cuda_check(I, cudaGetLastError(), "scatter"))) return rc;
    }
    return TL_OK;
}

int tl_update_pre_partials(tl_instance* inst, const tl_pre_op* ops, int count, int model) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    for (int k = 0; k < count; ++k)
        for (int c = 0; c < 2; ++c)
            if (ops[k].edge[c] >= 0)
                return fail(I, TL_ERR_ARG, "tl_update_pre_partials takes no edges (use "
                            "tl_pre_order_gradient)");
    int rc = pre_common(I, ops, count, model, 0, true, nullptr);
    if (rc) return rc;
    return cuda_check(I, cudaStreamSynchronize(I->stream), "tl_update_pre_partials");
}

int tl_pre_order_gradient(tl_instance* inst, const tl_pre_op* ops, int count, int model,
                          double* out_grad, int n_grad) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    if (!out_grad && n_grad > 0) return fail(I, TL_ERR_ARG, "out_grad is null");
    int rc;
    if ((rc = ensure_out(I, (size_t)2 * std::max(n_grad, 1) + 16))) return rc;
    double* d_g = extra(I).d_out + std::max(n_grad, 1) + 8;
    if ((rc = pre_common(I, ops, count, model, n_grad, false, d_g))) return rc;
    if (n_grad > 0)
        cudaMemcpyAsync(out_grad, d_g, sizeof(double) * n_grad, cudaMemcpyDeviceToHost, I->stream);
    if ((rc = cuda_check(I, cudaStreamSynchronize(I->stream), "tl_pre_order_gradient"))) return rc;
    return check_numeric_flag(I);
}

int tl_pre_order_derivative(tl_instance* inst, const tl_pre_op* ops, int count, int model,
                            double* out, int n_out) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    if (!out && n_out > 0) return fail(I, TL_ERR_ARG, "out is null");
    // the FP64 generic path always forms u . (dmat p) from the stored
    // derivative matrix, so it needs no switch for general derivatives
    int rc;
    if ((rc = ensure_out(I, (size_t)2 * std::max(n_out, 1) + 16))) return rc;
    double* d_g = extra(I).d_out + std::max(n_out, 1) + 8;
    if ((rc = pre_common(I, ops, count, model, n_out, false, d_g, 1))) return rc;
    if (n_out > 0)
        cudaMemcpyAsync(out, d_g, sizeof(double) * n_out, cudaMemcpyDeviceToHost, I->stream);
    if ((rc = cuda_check(I, cudaStreamSynchronize(I->stream), "tl_pre_order_derivative"))) return rc;
    return check_numeric_flag(I);
}

int tl_update_param_matrices(tl_instance* inst, int model, int param, const int* idx,
                             const double* edge_len, int count) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (model < 0 || model >= I->n_models || !I->models[model].ready)
        return fail(I, TL_ERR_STATE, "model %d not set", model);
    if (param < 0 || param >= I->models[model].n_dq)
        return fail(I, TL_ERR_INDEX, "model %d has %d parameters", model, I->models[model].n_dq);
    if (count < 0 || (count > 0 && (!idx || !edge_len))) return fail(I, TL_ERR_ARG, "bad arguments");
    for (int i = 0; i < count; ++i) {
        if (idx[i] < 0 || idx[i] >= I->n_mats) return fail(I, TL_ERR_INDEX, "idx[%d] out of range", i);
        if (!std::isfinite(edge_len[i]) || edge_len[i] < 0)
            return fail(I, TL_ERR_NUMERIC, "edge_len[%d] is negative or not finite", i);
    }
    if ((size_t)(I->R + count) > I->tmp_cap) {
        dev_free(I, I->d_tmp);
        I->tmp_cap = I->R + count + 1024;
        int rc = dev_alloc(I, &I->d_tmp, sizeof(double) * I->tmp_cap, "staging");
        if (rc) return rc;
    }
    int rc = stage(I, I->h_rates, I->R, edge_len, count);
    if (rc) return rc;
    void* d_idx = nullptr;
    if ((rc = upload(I, extra(I).areas[3], idx, sizeof(int) * count, &d_idx))) return rc;
    if ((rc = launch_param_matrices(I, model, param, (const int*)d_idx, I->d_tmp + I->R, count)))
        return rc;
    for (int i = 0; i < count; ++i) {
        I->mat_set[idx[i]] = 1;
        I->mat_model[idx[i]] = -1;
    }
    return TL_OK;
}

int tl_pre_order_gradient_dev(tl_instance* inst, const tl_pre_op* ops, int count, int model,
                              double* out_grad_dev, int n_grad) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    if (!out_grad_dev && n_grad > 0) return fail(I, TL_ERR_ARG, "out_grad_dev is null");
    return pre_common(I, ops, count, model, n_grad, false, out_grad_dev);
}

int tl_edge_derivatives(tl_instance* inst, const tl_edge* edges, int count, int model,
                        double* out_grad, int n_grad) {
    CHECK_INST(inst);
    Instance* I = reinterpret_cast<Instance*>(inst);
    if (int rc0 = activate_tip_pool(I)) return rc0;
    if (count < 0 || (count > 0 && !edges) || (n_grad > 0 && !out_grad))
        return fail(I, TL_ERR_ARG, "bad arguments");
    if (model < 0 || model >= I->n_models || !I->models[model].ready)
        return fail(I, TL_ERR_STATE, "model %d not set", model);
    if (use_tc(I)) return fail(I, TL_ERR_UNSUPPORTED, "edge derivatives not built for TL_PREC_TF32");
    std::vector<int> row(std::max(n_grad, 1), -1), map;
    std::vector<tl_edge> e(edges, edges + count);
    for (int k = 0; k < count; ++k) {
        const tl_edge& x = edges[k];
        if (x.post < 0 || x.post >= I->n_bufs || x.pre < I->n_tips || x.pre >= I->n_bufs)
            return fail(I, TL_ERR_INDEX, "edge %d: buffer out of range", k);
        if (x.post < I->n_tips ? !I->tip_set[x.post] : !I->buf_written[x.post - I->n_tips])
            return fail(I, TL_ERR_STATE, "edge %d: post buffer holds no data", k);
        if (!I->buf_written[x.pre - I->n_tips])
            return fail(I, TL_ERR_STATE, "edge %d: pre buffer holds no data", k);
        if (x.edge < 0 || x.edge >= n_grad) return fail(I, TL_ERR_INDEX, "edge %d: slot out of range", k);
        if (row[x.edge] >= 0) return fail(I, TL_ERR_ORDER, "edge slot %d requested twice", x.edge);
        row[x.edge] = (int)map.size();
        map.push_back(x.edge);
        e[k].edge = row[x.edge];
    }
    const int E = (int)map.size();
    int rc;
    int parts;
    if (use_nuc(I)) {
        parts = nuc_tiles(I);
        if ((rc = ensure_scratch(I, (size_t)std::max(E, 1) * parts))) return rc;
        std::vector<DevEdge> d(count);
        for (int k = 0; k < count; ++k) {
            const int b = e[k].post;
            const int kind = b < I->n_tips ? (I->tip_set[b] == 1 ? kTipStates : kTipPartials)
                                           : kInternal;
            d[k] = {b < I->n_tips ? b : b - I->n_tips, kind, e[k].pre - I->n_tips, e[k].edge};
        }
        void* d_e = nullptr;
        if ((rc = upload(I, extra(I).areas[2], d.data(), sizeof(DevEdge) * count, &d_e))) return rc;
        if ((rc = launch_edge4(I, (const DevEdge*)d_e, count, model, I->d_red))) return rc;
    } else {
        parts = generic_parts(I);
        if ((rc = ensure_scratch(I, (size_t)std::max(E, 1) * parts))) return rc;
        if ((rc = launch_edge_generic(I, e.data(), count, model, I->d_red, parts))) return rc;
    }
    if ((rc = ensure_out(I, (size_t)E + 1))) return rc;
    if ((rc = reduce_fixed(I, I->d_red, E, parts, extra(I).d_out))) return rc;
    std::vector<double> h(std::max(E, 1));
    if (E) cudaMemcpyAsync(h.data(), extra(I).d_out, sizeof(double) * E, cudaMemcpyDeviceToHost, I->stream);
    if ((rc = cuda_check(I, cudaStreamSynchronize(I->stream), "tl_edge_derivatives"))) return rc;
    for (int i = 0; i < n_grad; ++i) out_grad[i] = 0.0;
    for (int k = 0; k < E; ++k) out_grad[map[k]] = h[k];
    return TL_OK;
}


// ---------------------------------------------------------------------------
// batched four-state calls
// ---------------------------------------------------------------------------
namespace {

Batch* as_batch(tl_batch* b) { return reinterpret_cast<Batch*>(b); }

// Instances of a batched call: four-state FP32 or FP64, all of one precision
// and category count, on the batch's device, each at most once.
int batch_instances(Batch* B, tl_instance* const* insts, int n, std::vector<Instance*>* out) {
    if (n < 0 || (n > 0 && !insts)) return batch_fail(B, TL_ERR_ARG, "bad instance list");
    out->assign(n, nullptr);
    for (int k = 0; k < n; ++k) {
        Instance* I = reinterpret_cast<Instance*>(insts[k]);
        if (!I) return batch_fail(B, TL_ERR_ARG, "instance %d is null", k);
        if (!use_nuc(I))
            return batch_fail(B, TL_ERR_UNSUPPORTED,
                              "instance %d: batched calls take four-state FP32/FP64 instances", k);
        if (I->device != B->device)
            return batch_fail(B, TL_ERR_ARG, "instance %d is on device %d, the batch on %d", k,
                              I->device, B->device);
        if (k > 0 && (I->prec != (*out)[0]->prec || I->R != (*out)[0]->R))
            return batch_fail(B, TL_ERR_UNSUPPORTED,
                              "instance %d: precision or category count differs from instance 0", k);
        (*out)[k] = I;
    }
    std::vector<Instance*> sorted(*out);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
        return batch_fail(B, TL_ERR_ARG, "an instance appears twice in one batch");
    return TL_OK;
}

// An instance-level failure (validation, planning) reported on the batch.
int batch_from(Batch* B, Instance* I, int k, int rc) {
    return batch_fail(B, rc, "instance %d: %s", k, I->err.c_str());
}

// Batch stream after each instance stream's queued work (uploads, matrices).
int batch_order_before(Batch* B, const std::vector<Instance*>& I) {
    for (Instance* x : I) {
        if (x->stream == B->stream) continue;
        Extra& X = extra(x);
        cudaError_t e = cudaSuccess;
        if (!X.order_ev) e = cudaEventCreateWithFlags(&X.order_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(X.order_ev, x->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, X.order_ev, 0);
        if (e != cudaSuccess) return batch_cuda(B, e, "ordering before the batch");
    }
    return TL_OK;
}

// Each instance stream after the batched work (its buffers and scratch were
// in use on the batch stream).
int batch_order_after(Batch* B, const std::vector<Instance*>& I) {
    bool any = false;
    for (Instance* x : I) any = any || x->stream != B->stream;
    if (!any) return TL_OK;
    cudaError_t e = cudaSuccess;
    if (!B->done) e = cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(B->done, B->stream);
    for (Instance* x : I)
        if (e == cudaSuccess && x->stream != B->stream) e = cudaStreamWaitEvent(x->stream, B->done, 0);
    return batch_cuda(B, e, "ordering after the batch");
}

// One launch of fixed-order row sums for all jobs (area `which`).
int batch_reduce(Batch* B, int which, const std::vector<RedJob>& jobs) {
    const int n = (int)jobs.size();
    if (n == 0) return TL_OK;
    std::vector<int> begin(n + 1, 0);
    for (int k = 0; k < n; ++k) begin[k + 1] = begin[k] + jobs[k].n_out;
    const int total = begin[n];
    if (total == 0) return TL_OK;
    const size_t hdr = (((size_t)(n + 1) * sizeof(int) + 15) / 16) * 16;
    std::vector<unsigned char> buf(hdr + sizeof(RedJob) * n, 0);
    std::memcpy(buf.data(), begin.data(), sizeof(int) * (n + 1));
    std::memcpy(buf.data() + hdr, jobs.data(), sizeof(RedJob) * n);
    void* d = nullptr;
    int rc = batch_upload(B, which, buf.data(), buf.size(), &d);
    if (rc) return rc;
    const int* d_begin = static_cast<const int*>(d);
    const RedJob* d_jobs = reinterpret_cast<const RedJob*>(static_cast<unsigned char*>(d) + hdr);
    k_reduce_batch<<<(total + kRedWarps - 1) / kRedWarps, kRedWarps * 32, 0, B->stream>>>(
        d_jobs, d_begin, n, total);
    B->launches += 1;
    return batch_cuda(B, cudaGetLastError(), "batched reduction");
}

}  // namespace

int tl_batch_create(void* stream, tl_batch** out) {
    if (!out) return fail(nullptr, TL_ERR_ARG, "out is null");
    *out = nullptr;
    Batch* B = new Batch();
    B->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&B->device);
    if (e != cudaSuccess) {
        delete B;
        return cuda_check(nullptr, e, "tl_batch_create");
    }
    *out = reinterpret_cast<tl_batch*>(B);
    return TL_OK;
}

int tl_batch_destroy(tl_batch* b) {
    if (!b) return TL_ERR_ARG;
    Batch* B = as_batch(b);
    cudaStreamSynchronize(B->stream);
    for (auto& A : B->areas)
        if (A.d) cudaFree(A.d);
    for (auto& s : B->ring) {
        if (s.h) cudaFreeHost(s.h);
        if (s.ev) cudaEventDestroy(s.ev);
    }
    if (B->done) cudaEventDestroy(B->done);
    delete B;
    return TL_OK;
}

int tl_batch_last_error(const tl_batch* b, char* buf, size_t len) {
    if (!buf || len == 0) return TL_ERR_ARG;
    const std::string& s = b ? reinterpret_cast<const Batch*>(b)->err : g_create_err;
    size_t n = std::min(len - 1, s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
    return TL_OK;
}

int tl_batch_launch_count(const tl_batch* b, unsigned long long* out) {
    if (!b || !out) return TL_ERR_ARG;
    *out = reinterpret_cast<const Batch*>(b)->launches;
    return TL_OK;
}

int tl_batch_update_partials(tl_batch* b, tl_instance* const* insts, const tl_op* const* ops,
                             const int* counts, int n) {
    if (!b) return fail(nullptr, TL_ERR_ARG, "null batch");
    Batch* B = as_batch(b);
    std::vector<Instance*> I;
    int rc = batch_instances(B, insts, n, &I);
    if (rc) return rc;
    if (n > 0 && !counts) return batch_fail(B, TL_ERR_ARG, "counts is null");
    std::vector<const DevPostOp*> d_ops(n, nullptr);
    std::vector<int> n_ops(n, 0), n_slots(n, 0);
    for (int k = 0; k < n; ++k) {
        if (counts[k] < 0 || (counts[k] > 0 && (!ops || !ops[k])))
            return batch_fail(B, TL_ERR_ARG, "instance %d: bad op list", k);
        if (counts[k] == 0) continue;
        PostPlan plan;
        if ((rc = plan_post(I[k], ops[k], counts[k], &plan, false))) return batch_from(B, I[k], k, rc);
        void* d = nullptr;
        if ((rc = upload(I[k], extra(I[k]).areas[0], plan.dev.data(),
                         sizeof(DevPostOp) * counts[k], &d)))
            return batch_from(B, I[k], k, rc);
        d_ops[k] = static_cast<const DevPostOp*>(d);
        n_ops[k] = counts[k];
        n_slots[k] = plan.n_slots;
    }
    if ((rc = batch_order_before(B, I))) return rc;
    if ((rc = nuc_batch_post(B, I.data(), d_ops.data(), n_ops.data(), n_slots.data(), n))) return rc;
    if ((rc = batch_order_after(B, I))) return rc;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < counts[k]; ++j) I[k]->buf_written[ops[k][j].dest - I[k]->n_tips] = 1;
    return TL_OK;
}

int tl_batch_root_loglik_dev(tl_batch* b, tl_instance* const* insts, const int* roots,
                             const int* models, int n, double* out_logl_dev) {
    if (!b) return fail(nullptr, TL_ERR_ARG, "null batch");
    Batch* B = as_batch(b);
    std::vector<Instance*> I;
    int rc = batch_instances(B, insts, n, &I);
    if (rc) return rc;
    if (n == 0) return TL_OK;
    if (!roots || !models || !out_logl_dev) return batch_fail(B, TL_ERR_ARG, "null argument");
    std::vector<int> kind(n), idx(n);
    std::vector<double*> part(n);
    std::vector<RedJob> red(n);
    for (int k = 0; k < n; ++k) {
        Instance* x = I[k];
        const int root = roots[k], model = models[k];
        if (root < 0 || root >= x->n_bufs)
            return batch_fail(B, TL_ERR_INDEX, "instance %d: root %d out of range", k, root);
        if (root >= x->n_tips ? !x->buf_written[root - x->n_tips] : !x->tip_set[root])
            return batch_fail(B, TL_ERR_STATE, "instance %d: root buffer %d holds no data", k, root);
        if (model < 0 || model >= x->n_models || !x->models[model].ready)
            return batch_fail(B, TL_ERR_STATE, "instance %d: model %d not set", k, model);
        const int n_tiles = nuc_tiles(x);
        if ((rc = ensure_scratch(x, n_tiles))) return batch_from(B, x, k, rc);
        kind[k] = kInternal;
        idx[k] = root - x->n_tips;
        if (root < x->n_tips) {
            kind[k] = x->tip_set[root] == 1 ? kTipStates : kTipPartials;
            idx[k] = root;
        }
        part[k] = x->d_red;
        red[k] = RedJob{x->d_red, nullptr, out_logl_dev + k, n_tiles, 1};
    }
    if ((rc = batch_order_before(B, I))) return rc;
    if ((rc = nuc_batch_root(B, I.data(), kind.data(), idx.data(), models, n, part.data())))
        return rc;
    if ((rc = batch_reduce(B, 3, red))) return rc;
    return batch_order_after(B, I);
}

int tl_batch_pre_order_gradient_dev(tl_batch* b, tl_instance* const* insts,
                                    const tl_pre_op* const* ops, const int* counts,
                                    const int* models, double* const* out_grad_dev,
                                    const int* n_grad, int n) {
    if (!b) return fail(nullptr, TL_ERR_ARG, "null batch");
    Batch* B = as_batch(b);
    std::vector<Instance*> I;
    int rc = batch_instances(B, insts, n, &I);
    if (rc) return rc;
    if (n == 0) return TL_OK;
    if (!counts || !models || !out_grad_dev || !n_grad)
        return batch_fail(B, TL_ERR_ARG, "null argument");
    std::vector<const DevPreOp*> d_ops(n, nullptr);
    std::vector<int> n_ops(n, 0), n_slots(n, 0);
    std::vector<double*> gpart(n);
    std::vector<RedJob> red;
    for (int k = 0; k < n; ++k) {
        Instance* x = I[k];
        if (counts[k] < 0 || (counts[k] > 0 && (!ops || !ops[k])))
            return batch_fail(B, TL_ERR_ARG, "instance %d: bad op list", k);
        if (models[k] < 0 || models[k] >= x->n_models || !x->models[models[k]].ready)
            return batch_fail(B, TL_ERR_STATE, "instance %d: model %d not set", k, models[k]);
        if (n_grad[k] < 0) return batch_fail(B, TL_ERR_ARG, "instance %d: n_grad < 0", k);
        if (n_grad[k] > 0 && !out_grad_dev[k])
            return batch_fail(B, TL_ERR_ARG, "instance %d: output is null", k);
        PrePlan plan;
        if ((rc = plan_pre(x, ops ? ops[k] : nullptr, counts[k], n_grad[k], false, &plan)))
            return batch_from(B, x, k, rc);
        const int E = (int)plan.edge_map.size();
        const int n_tiles = nuc_tiles_pre(x);
        if ((rc = ensure_scratch(x, (size_t)std::max(E, 1) * n_tiles))) return batch_from(B, x, k, rc);
        void* d = nullptr;
        if (counts[k] > 0 &&
            (rc = upload(x, extra(x).areas[1], plan.dev.data(), sizeof(DevPreOp) * counts[k], &d)))
            return batch_from(B, x, k, rc);
        d_ops[k] = static_cast<const DevPreOp*>(d);
        n_ops[k] = counts[k];
        n_slots[k] = plan.n_slots;
        gpart[k] = x->d_red;
        if (n_grad[k] > 0) {
            // out[g] = row inv[g] of the gradient partials, 0 for slots no op names
            std::vector<int> inv(n_grad[k], -1);
            for (int e = 0; e < E; ++e) inv[plan.edge_map[e]] = e;
            void* d_inv = nullptr;
            if ((rc = upload(x, extra(x).areas[5], inv.data(), sizeof(int) * inv.size(), &d_inv)))
                return batch_from(B, x, k, rc);
            red.push_back(RedJob{x->d_red, static_cast<const int*>(d_inv), out_grad_dev[k], n_tiles,
                                 n_grad[k]});
        }
    }
    if ((rc = batch_order_before(B, I))) return rc;
    if ((rc = nuc_batch_pre(B, I.data(), d_ops.data(), n_ops.data(), n_slots.data(), models,
                            gpart.data(), n)))
        return rc;
    if ((rc = batch_reduce(B, 4, red))) return rc;
    return batch_order_after(B, I);
}

}  // extern "C"

namespace tl {
int upload_bytes(Instance* I, void* dst, const void* src, size_t bytes) {
    return h2d(I, dst, src, bytes);
}

int batch_fail(Batch* B, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (B) B->err = buf;
    else g_create_err = buf;
    return code;
}

int batch_cuda(Batch* B, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TL_OK;
    return batch_fail(B, e == cudaErrorMemoryAllocation ? TL_ERR_OOM : TL_ERR_CUDA, "%s: %s (%s)",
                      what, cudaGetErrorString(e), cudaGetErrorName(e));
}

int batch_upload(Batch* B, int which, const void* src, size_t bytes, void** dptr) {
    Batch::Area& A = B->areas[which];
    cudaError_t e = cudaSuccess;
    if (A.cap < bytes) {
        if (A.d) {
            cudaStreamSynchronize(B->stream);
            cudaFree(A.d);
            A.d = nullptr;
            A.cap = 0;
        }
        const size_t cap = std::max<size_t>(bytes * 2, 4096);
        e = cudaMalloc(&A.d, cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            A.d = nullptr;
            return batch_cuda(B, e, "batch table");
        }
        A.cap = cap;
    }
    Batch::Slot& s = B->ring[B->ring_next];
    B->ring_next = (B->ring_next + 1) % Batch::kSlots;
    if (s.ev) e = cudaEventSynchronize(s.ev);
    else e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return batch_cuda(B, e, "staging event");
    if (s.cap < bytes) {
        if (s.h) cudaFreeHost(s.h);
        s.cap = std::max<size_t>(bytes, 64 * 1024);
        e = cudaHostAlloc(&s.h, s.cap, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            s.h = nullptr;
            s.cap = 0;
            return batch_cuda(B, e, "pinned staging");
        }
    }
    std::memcpy(s.h, src, bytes);
    e = cudaMemcpyAsync(A.d, s.h, bytes, cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.ev, B->stream);
    *dptr = A.d;
    return batch_cuda(B, e, "batch table copy");
}
}  // namespace tl
