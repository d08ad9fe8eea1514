// Internal declarations of the treelik library (device structs, instance
// state and the launchers each translation unit exports).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "treelik.h"

namespace tl {

constexpr int kWarpsPerBlock = 4;
constexpr int kMaxCat = 8;
constexpr int kMaxStates = 64;
constexpr int kMaxDq = 8;      // dQ/dtheta matrices kept per model
constexpr int kColStride = 5;  // four-state matrices: 4 columns + row sums
constexpr int kPadPatterns = 64;  // patterns are padded to a multiple of this

enum Prec { kF64 = 0, kF32 = 1, kTF32 = 2, kBF16X3 = 3 };

// Where a four-state kernel finds a child's partials.
enum ChildKind { kInternal = 0, kTipStates = 1, kTipPartials = 2 };
// On-chip sources of an op input (>= 0 is a shared-memory slot).
constexpr int kFromMemory = -1;
constexpr int kFromRegisters = -2;  // the result of the op just before
constexpr int kFromRoot = -3;       // pre-order: q = pi

// One post-order op as the device walks it. Buffer indices are relative to
// the internal partials pool; tips are indexed 0..n_tips-1.
struct __align__(16) DevPostOp {
    int child[2];
    int kind[2];
    int mat[2];
    int slot_in[2];  // kFromMemory, kFromRegisters or a slot
    int dest;
    int slot_out;    // slot receiving dest (-1: none)
    int store;       // 1: write dest to its buffer
    int pad;
};

// One pre-order op (one parent, both children) as the device walks it. The
// first 16 bytes (children and their kinds) are what the kernels prefetch.
struct __align__(16) DevPreOp {
    int child[2];
    int kind[2];
    int q_src;       // kFromRoot, kFromRegisters, kFromMemory or a slot
    int q_reg;       // which q output (0, 1) the next op takes from registers (-1: none)
    int q_buf_in;    // with kFromMemory: pool index of q
    int mat[2];
    int dmat[2];     // -1: no derivative
    int q_slot_out[2];
    int q_buf_out[2];  // pool index or -1
    int edge[2];     // row of the gradient partials or -1
    int need_q[2];
    int pad;
};

struct __align__(16) DevEdge {
    int post;        // pool index, or tip index
    int kind;
    int pre;         // pool index
    int edge;
};

// Arguments of the four-state kernels, passed by value. Partials of
// internal buffer b live at pool + b * bstride as [R][Ppad][4]; its
// accumulated exponents at epool + b * Ppad; tip t's states at
// tips + t * Ppad.
template <typename T>
struct NucArgs {
    T* pool;
    int* epool;
    const int8_t* tips;
    T* const* tipbuf;               // device table: tip partials (kind 2)
    const T* mat;                   // [mat][5 columns][R][4] working copies
    const double* patw;             // [Ppad] pattern weights (0 on padding)
    size_t bstride;
    int P, Ppad, R, n_slots, rescale, mat_stride, n_tiles;
    T catw[kMaxCat];
    T rates[kMaxCat];
};

// One instance's share of a batched four-state launch: its kernel
// arguments, op list and outputs, and the first tile of the launch's global
// tile range that belongs to it (tiles are handed out in global order).
template <typename T>
struct __align__(16) BatchJob {
    NucArgs<T> a;         // a.n_tiles: this job's tiles
    const void* ops;      // DevPostOp or DevPreOp list
    const T* piw;         // pre-order: pi and Q of the job's model (working precision)
    const T* Qw;
    double* gpart;        // pre-order: [edge][a.n_tiles] gradient partials
    const double* pi;     // root: pi (FP64)
    double* part;         // root: [a.n_tiles] partial sums
    int* err;             // root: the instance's numeric-error flag
    int n_ops;
    int root_kind, root;  // root: the buffer and its kind
    int pad;
};

// The job table of a batched launch: jobs[j] owns global tiles
// [tile_begin[j], tile_begin[j + 1]); warps claim tiles from *counter.
template <typename T>
struct BatchRef {
    const BatchJob<T>* jobs;
    const int* tile_begin;
    int* counter;
    int n_jobs;
};

// One job of a batched fixed-order reduction: out[g] = sum of the n_in
// doubles of row inv[g] of `in` (row g when inv is null; 0 when inv[g] < 0),
// for g < n_out.
struct __align__(16) RedJob {
    const double* in;
    const int* inv;
    double* out;
    int n_in, n_out;
};

struct ModelDev {
    double* Q = nullptr;      // [Spad][Spad]
    double* pi = nullptr;     // [Spad]
    double* V = nullptr;      // [Spad][Spad]
    double* Vinv = nullptr;   // [Spad][Spad]
    double* lam = nullptr;    // [Spad]
    double* dQ = nullptr;     // [kMaxDq][Spad][Spad]
    double* G = nullptr;      // [kMaxDq][Spad][Spad]: Vinv dQ V, then as much scratch
    void* piw = nullptr;      // pi in working precision [Spad]
    void* Qw = nullptr;       // Q in working precision [Spad][Spad]
    void* Vdf = nullptr;      // reduced precision: V and Vinv as double-float pairs
    void* Vinvdf = nullptr;   // (two floats per entry) [Spad][Spad] for the matrix products
    int* pairs = nullptr;     // GY94RE: [TL_GY94_PAIRS][2] codon indices (i < j)
    double* mu = nullptr;     // [1] mean rate of the unnormalised Q (tl_set_model)
    int n_dq = 0;
    int kind = 0;             // TL_MODEL_* (0: set from Q or an eigensystem)
    int n_params = 0;         // parameters of tl_set_model
    bool ready = false;
    bool basis_ready = false;  // G computed for the current V, Vinv, dQ
};

struct Instance {
    int n_tips = 0, P = 0, Ppad = 0, S = 0, Spad = 0, R = 0;
    int n_buffers = 0, n_mats = 0, n_models = 0;
    int n_bufs = 0;  // n_tips + n_buffers
    unsigned flags = 0;
    Prec prec = kF64;
    int elt = 8;      // bytes per stored partial element
    int rescale = 1;
    int split = 0;    // TF32: matrices as hi + lo (TL_SPLIT_MATRICES)
    int split_partials = 0;  // TF32: FP32 partials split on chip (TL_SPLIT_PARTIALS)
    cudaStream_t stream = nullptr;
    int device = 0;
    int smem_optin = 0;

    // device memory
    void* pool = nullptr;            // internal partials
    int* scale_pool = nullptr;       // [n_buffers][Ppad]
    std::vector<void*> tip_part;     // per-tip partials allocations
    int8_t* tip_pool = nullptr;      // [n_tips][Ppad] tip states (pad: ambiguous)
    void** d_buf = nullptr;          // device table [n_bufs]
    int** d_scale = nullptr;         // device table [n_bufs]
    int8_t** d_tipst = nullptr;      // device table [n_tips]
    std::vector<void*> h_buf;        // host mirrors
    std::vector<int*> h_scale;
    std::vector<int8_t*> h_tipst;
    std::vector<char> tip_set;       // 0 unset, 1 states, 2 partials
    std::vector<char> buf_written;   // internal buffer holds post data
    double* d_patw = nullptr;
    double* h_catw = nullptr;        // host copies [kMaxCat]
    double* h_rates = nullptr;
    double* d_mat64 = nullptr;       // FP64 master matrices [n_mats][R][Spad][Spad]
    void* d_matw = nullptr;          // working copies
    size_t matw_stride = 0;          // elements per matrix slot in d_matw
    std::vector<char> mat_set;
    std::vector<double> mat_len;     // length each P slot was last computed with
    std::vector<int> mat_model;      // and its model (-1: not a P, or a derivative)
    std::vector<ModelDev> models;

    // scratch
    double* d_red = nullptr;         // reduction partials
    size_t red_cap = 0;              // doubles
    int* d_err = nullptr;            // device error flags [4]
    void* d_ops = nullptr;           // op list upload area
    size_t ops_cap = 0;              // bytes
    std::vector<char> last_ops;      // bytes last uploaded (skip identical uploads)
    double* d_tmp = nullptr;         // small staging (params, lengths)
    size_t tmp_cap = 0;
    void* host_extra = nullptr;      // host-side helper state (tl_api.cu)
    // tensor-core (TF32) instances
    float* d_rowsum = nullptr;       // [mat][R][64] row sums of the rounded P
    float* tc_tip_pool = nullptr;    // [n_tips][R][Ppad][64] tip partials (lazy)
    std::vector<unsigned char> tmaps;  // CUtensorMap x3: pool, tip pool, matrices

    size_t bytes = 0;
    unsigned long long launches = 0; // kernels this instance has launched
    std::string err;
};

// A batch context: a stream, device areas for job tables and a pinned
// staging ring, shared by the batched calls (tl_api.cu).
struct Batch {
    struct Area {
        void* d = nullptr;
        size_t cap = 0;
    };
    struct Slot {
        void* h = nullptr;
        size_t cap = 0;
        cudaEvent_t ev = nullptr;
    };
    static constexpr int kAreas = 8, kSlots = 8;
    cudaStream_t stream = nullptr;
    int device = 0;
    Area areas[kAreas];
    Slot ring[kSlots];
    int ring_next = 0;
    cudaEvent_t done = nullptr;  // instance streams wait on this after a batched call
    unsigned long long launches = 0;
    std::string err;
};
// Copy bytes to device area `which` of the batch (grown as needed) through
// the pinned ring, on the batch stream; *dptr receives the area.
int batch_upload(Batch* B, int which, const void* src, size_t bytes, void** dptr);
int batch_fail(Batch* B, int code, const char* fmt, ...);
int batch_cuda(Batch* B, cudaError_t e, const char* what);

// ---- launchers (one translation unit each) --------------------------------
// tl_model.cu
int launch_build_model(Instance* I, int m, int kind, const double* d_params, int n_params,
                       const double* d_freqs, int n_freqs, bool check);
int launch_eigen_from_q(Instance* I, int m, bool check);  // Q, pi already in the slot
int launch_q_from_eigen(Instance* I, int m);  // V, Vinv, lambda already in the slot
int launch_model_working_copies(Instance* I, int m);
int launch_update_matrices(Instance* I, int m, const int* d_pidx, const int* d_dpidx,
                           const double* d_len, int count);
int launch_param_matrices(Instance* I, int m, int param, const int* d_idx, const double* d_len,
                          int count);

// tl_nuc.cu (four-state pattern-tile kernels, T = float or double)
int nuc_lanes(const Instance* I);            // lanes per pattern (root, edge kernels)
int nuc_tiles(const Instance* I);            // their tiles
int nuc_lanes_main(const Instance* I);       // lanes per pattern (post, pre kernels)
int nuc_tiles_main(const Instance* I);       // their tiles
int nuc_lanes_pre(const Instance* I);        // lanes per pattern (pre-order kernel)
int nuc_tiles_pre(const Instance* I);        // its tiles (= gradient partial columns)
int nuc_smem_per_slot(const Instance* I);    // bytes per slot per warp and pattern per lane
int nuc_post_ppl(const Instance* I);         // patterns per lane (post-order kernel)
int nuc_pre_slot_cap(const Instance* I);     // on-chip q slots of the pre-order kernel
int launch_post4(Instance* I, const DevPostOp* d_ops, int n_ops, int n_slots);
int launch_root4(Instance* I, int root_kind, int root, int model, double* d_site,
                 double* d_part);
int launch_pre4(Instance* I, const DevPreOp* d_ops, int n_ops, int n_slots, int model,
                double* d_gpart, int dgen);
int launch_edge4(Instance* I, const DevEdge* d_edges, int n_edges, int model, double* d_gpart);

// batched four-state launches over several instances of one precision and
// category count (tl_batch.cu builds the job tables)
struct Batch;
int nuc_batch_post(Batch* B, Instance* const* I, const DevPostOp* const* d_ops, const int* n_ops,
                   const int* n_slots, int n);
int nuc_batch_root(Batch* B, Instance* const* I, const int* kind, const int* root,
                   const int* model, int n, double* const* d_part);
int nuc_batch_pre(Batch* B, Instance* const* I, const DevPreOp* const* d_ops, const int* n_ops,
                  const int* n_slots, const int* model, double* const* d_gpart, int n);

// tl_generic.cu (FP64, any S)
int launch_post_generic(Instance* I, const tl_op* h_ops, int n_ops);
int launch_root_generic(Instance* I, int root, int model, double* d_site, double* d_part,
                        int n_parts);
int launch_pre_generic(Instance* I, const tl_pre_op* h_ops, int n_ops, int model,
                       double* d_gpart, int n_parts);
int launch_edge_generic(Instance* I, const tl_edge* h_edges, int n_edges, int model,
                        double* d_gpart, int n_parts);
int generic_parts(const Instance* I);
struct EigOp {             // one post-order op with its children's edge lengths
    int dest, child[2], pad;
    double len[2];
};
int launch_post_eig(Instance* I, int model, const EigOp* d_ops, const int* level_start,
                    int n_levels);

// tl_codon_tc.cu (tcgen05 codon path)
constexpr size_t kTcOpBytes = 64;  // one tensor-core work descriptor
int tc_tile();
int tc_setup(Instance* I);
int tc_set_tip_pool(Instance* I);
int launch_post_tc(Instance* I, const tl_op* ops, int n, void* d_ops_area, size_t cap);
int tc_fused_enabled(const Instance* I);   // subtree-fused post-order kernel in use
int launch_post_tc_fused(Instance* I, const DevPostOp* plan_ops, int n, void* d_ops_area,
                         size_t cap);
int launch_root_tc(Instance* I, int root_pool, int model, double* d_site, double* d_part,
                   int n_parts);
int launch_pre_tc(Instance* I, const tl_pre_op* ops, int n, const int* edge_row, int model,
                  double* d_gpart, void* d_ops_area, size_t cap, int dgen);
int launch_q_tc(Instance* I, int model);
size_t tc_matw_floats(const Instance* I);

// tl_adjoint.cu (reverse-mode adjoint): one parent as the device reads it.
// Partials are [R][Ppad][Spad] in the working precision; a tip with states
// has part == nullptr and st set; exponents are cumulative (nullptr: 0).
template <typename T>
struct __align__(16) AdjOp {
    const T* q;            // parent's pre-order partial; nullptr at the root (q = pi)
    const T* pn;           // parent's post-order partial
    const int* en;         // its cumulative exponents
    const T* part[2];      // children's partials (nullptr: tip states)
    const int* ec[2];      // children's cumulative exponents (nullptr: 0)
    const int8_t* st[2];   // children's tip states
    const double* P[2];    // FP64 transition matrices of the edges [R][Spad][Spad]
    int row[2];            // output row of each edge (-1: not listed)
};
struct AdjArgs {
    const double* pi;     // [Spad]
    const double* patw;   // [Ppad]
    const double* coef;   // generic path: [n_ops][Ppad] w_p / L_p (scaled)
    int* err;             // numeric flag (zero pattern likelihood)
    int* timeout;         // tensor-core wait flag (bit 11: the adjoint kernel)
    int R, Ppad, Spad, S, chunk, n_chunks;
    size_t n_rows;        // rows of the per-chunk outputs: listed edges x R x Spad^2
    double catw[kMaxCat];
};
// tl_adjoint_tc.cu: both accumulation products of a TF32 instance (Spad 64)
// on the 5th-generation tensor cores
int launch_adj_tc(Instance* I, const AdjOp<float>* d_ops, int n_ops, int n_chunks,
                  const AdjArgs& a, double* d_mpart);
struct AdjEdge {           // one listed edge for the eigenbasis finish
    const double* P;       // [R][Spad][Spad]
    double t;
};
int adj_chunks(const Instance* I, int n_ops);
int launch_adj_accumulate(Instance* I, const void* d_ops, int n_ops, int n_chunks, size_t n_rows,
                          double* d_coef, double* d_mpart, int model);
int launch_adj_sum_chunks(Instance* I, const double* d_in, size_t n_rows, int n_chunks,
                          double* d_out);
int launch_adj_finish(Instance* I, int model, const double* d_M, const AdjEdge* d_edges, int E,
                      bool first_order, double* d_gpart, double* d_grad);
int launch_adj_params(Instance* I, int model, const double* d_G, bool first_order, double* d_dQ,
                      double* d_theta);

// tl_ratio.cu: the node-height ratio transform (host arrays in and out)
int ratio_run(int n_tips, const int* parent, const double* tip_h, const double* ratio,
              double root_h, const double* rate, const double* grad, double* out_h,
              double* out_len, double* out_gr, double* out_groot, double* out_grate,
              void* stream, std::string* err);

// tl_api.cu helpers used by the other units
int upload_bytes(Instance* I, void* dst, const void* src, size_t bytes);
int fail(Instance* I, int code, const char* fmt, ...);
int cuda_check(Instance* I, cudaError_t e, const char* what);
int reduce_fixed(Instance* I, const double* d_in, int n_out, int n_in, double* d_out);

}  // namespace tl
