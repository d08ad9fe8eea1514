/*
 * treelik -- C ABI of the GB300 (sm_103a) phylogenetic likelihood library.
 *
 * Computes the log-likelihood of aligned sequence data on a rooted binary
 * tree by Felsenstein pruning (post-order partial likelihoods) and its
 * gradient by the linear-time pre-order scheme of the paper (Sec.
 * "Algorithmic advances": post- and pre-order partials whose inner product
 * is the likelihood; Sec. "Discussion": the branch-length gradient is a
 * sandwich of a pre-order partial, the rate matrix and a post-order partial;
 * transition matrices come from an eigendecomposition of Q, cached across
 * patterns, or formed inside pruning for single-pattern problems; exact
 * substitution-parameter gradients through the adjoint of the matrix
 * exponential; random-effects models; the node-height ratio transform).
 *
 * Conventions shared by every call
 *  - Every function returns an int status: TL_OK (0) or a negative TL_ERR_*
 *    code; tl_last_error() gives the text of the instance's last error.
 *    No C++ exception crosses this boundary.
 *  - Host arrays passed in are borrowed for the duration of the call and
 *    copied; the caller keeps ownership. Results written to host pointers
 *    are complete when the call returns (the call synchronises the
 *    instance's stream). Calls whose name ends in _dev take and return
 *    device pointers and do not synchronise.
 *  - The instance owns all of its device memory (partials, matrices,
 *    scratch) and frees it in tl_destroy. All device work is enqueued on the
 *    CUDA stream given at creation (NULL = the legacy default stream).
 *  - An instance is not thread-safe; use one instance per host thread.
 *  - Buffer indices: 0 .. n_tips-1 name the tips; n_tips ..
 *    n_tips+n_buffers-1 name internal partials buffers (post- or pre-order).
 *    Matrix slots are 0 .. n_matrices-1; model slots 0 .. n_models-1.
 *  - Layouts: host matrices are row-major S x S doubles; tip states are one
 *    int8 code per pattern; tip partials are [pattern][state] doubles.
 *    Device partials are [category][pattern][state] in the instance's
 *    working precision, patterns padded to a multiple of 64 (128 for
 *    TL_PREC_TF32), states to a multiple of 4 (64 for TL_PREC_TF32).
 */
#ifndef TREELIK_H
#define TREELIK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TL_OK               0
#define TL_ERR_ARG         -1  /* bad argument (size, null pointer, flag)      */
#define TL_ERR_INDEX       -2  /* buffer / matrix / model index out of range   */
#define TL_ERR_ORDER       -3  /* op list reads a buffer it writes later, or
                                  writes one buffer twice                      */
#define TL_ERR_OOM         -4  /* device allocation failed                     */
#define TL_ERR_NUMERIC     -5  /* a pattern likelihood is zero, negative or
                                  not finite, or an input is not finite        */
#define TL_ERR_TIMEOUT     -6  /* a bounded device wait gave up                */
#define TL_ERR_CUDA        -7  /* a CUDA runtime call failed                   */
#define TL_ERR_UNSUPPORTED -8  /* combination of sizes/precision not built     */
#define TL_ERR_STATE       -9  /* required input not set yet (model, matrix)   */

/* ---- creation flags ---------------------------------------------------- */
#define TL_PREC_F64    0x1u   /* FP64 partials and matrices (any S <= 64)      */
#define TL_PREC_F32    0x2u   /* FP32 partials (S == 4), FP64 reductions       */
#define TL_PREC_TF32   0x4u   /* S in 5..64: tcgen05 kind::tf32 contractions,
                                 TF32-rounded FP32 partials, FP32 accumulate   */
#define TL_PREC_BF16X3 0x8u   /* reserved for a BF16 hi/lo split (three
                                 products per contraction); not built:
                                 tl_create returns TL_ERR_UNSUPPORTED          */
#define TL_SCALE_NONE  0x100u /* no per-pattern rescaling (FP64 only)          */
#define TL_SPLIT_MATRICES 0x200u /* with TL_PREC_TF32: every transition matrix
                                 (and Q, dP) is the exact FP32 sum of two TF32
                                 terms, hi + lo, and each contraction is two
                                 tensor-core products (x.P_hi + x.P_lo). The
                                 stored partials are TF32 values already, so
                                 a split of them would add nothing; the split
                                 removes the matrix rounding, the one error
                                 shared by all patterns (it would not average
                                 out over the pattern sum). */
#define TL_SPLIT_PARTIALS 0x400u /* with TL_PREC_TF32 | TL_SPLIT_MATRICES:
                                 partials are stored in full FP32 and every
                                 tensor-core operand tile of partials is
                                 split on chip into TF32 hi + lo (hi the
                                 truncation, lo the truncation of the rest);
                                 each contraction is three products
                                 (x_hi P_hi + x_hi P_lo + x_lo P_hi), about
                                 21 bits of both operands, so logL and every
                                 gradient component carry FP32-level errors
                                 (the per-pattern TF32 rounding of stored
                                 partials is what limits the gradient of the
                                 two modes above) */

/* ---- model kinds for tl_set_model -------------------------------------- */
#define TL_MODEL_HKY   1  /* S=4.  params: kappa.  freqs: pi[4]                */
#define TL_MODEL_GTR   2  /* S=4.  params: AC,AG,AT,CG,CT,GT.  freqs: pi[4]    */
#define TL_MODEL_GY94  3  /* S=61. params: kappa, omega.  freqs: F3x4 [3][4]   */
#define TL_MODEL_REV   4  /* any S. params: symmetric S x S exchangeabilities
                             (row-major, diagonal ignored).  freqs: pi[S]      */
#define TL_MODEL_GY94RE 5 /* S=61. GY94 with a multiplicative random effect on
                             every non-zero off-diagonal element (Sec.
                             "Algorithmic advances": random-effects models),
                             s_ij = s_ji scaled by exp(eps_k) so Q stays
                             reversible. params: kappa, omega, then eps_k for
                             the TL_GY94_PAIRS unordered pairs (i < j) of sense
                             codons that differ at one position, in
                             lexicographic (i, j) order (any real eps).
                             freqs: F3x4 [3][4]. dQ/dtheta is kept for kappa
                             and omega; tl_adjoint returns all 265.         */
#define TL_GY94_PAIRS 263

typedef struct tl_instance tl_instance;

/* Post-order partials update (Sec. "Introduction", Felsenstein pruning):
 *   dest[r,p,:] = (P_mat1,r child1[r,p,:]) o (P_mat2,r child2[r,p,:])
 * then rescaled per pattern by a power of two (unless TL_SCALE_NONE); the
 * removed exponents of the whole subtree are kept with dest. A child that is
 * a tip with states uses a column lookup of P instead of a product. */
typedef struct {
    int dest;
    int child1, mat1;
    int child2, mat2;
} tl_op;

/* Pre-order step for one parent node (Sec. "Algorithmic advances"). For
 * each child c (sibling s) with post-order partial p_c:
 *   u_c = q_parent o (P_s p_s),   q_c = P_c^T u_c   (rescaled per pattern)
 * q_parent is the pre-order partial of the parent: buffer parent_pre, or the
 * root distribution pi when parent_pre == -1. pre_c >= 0 names the buffer
 * that receives q_c (-1: q_c is not needed). edge_c >= 0 is the slot of
 * out_grad that receives dlogL/dt_c, computed from dmat_c = dP/dt (see
 * tl_update_matrices) as
 *   sum_p w_p [sum_r w_r u_c^T dP_c p_c] / [sum_r w_r u_c^T P_c p_c]
 * (Sec. "Discussion": pre-order partial . dP/dt . post-order partial). */
typedef struct {
    int parent_pre;
    int child[2];
    int mat[2];
    int dmat[2];
    int pre[2];
    int edge[2];
} tl_pre_op;

/* One edge for tl_edge_derivatives: post-order partial p_c (buffer or tip),
 * materialised pre-order partial q_c (buffer), and the slot of out_grad. */
typedef struct {
    int post;
    int pre;
    int edge;
} tl_edge;

/* Create an instance. n_states: 1..64 (TL_PREC_F32: 4; TF32: 5..64, stored
 * padded to 64, e.g. 20 amino acids or 61 codons). n_categories: 1..8 (TL_PREC_TF32: 1..4; more
 * returns TL_ERR_UNSUPPORTED). n_buffers: internal partials
 * buffers. n_matrices: transition-matrix slots (each holds all categories).
 * n_models: model slots (Q, pi, eigensystem, dQ/dtheta). stream: a
 * cudaStream_t or NULL. Exactly one TL_PREC_* flag must be set. */
int tl_create(int n_tips, int n_patterns, int n_states, int n_categories,
              int n_buffers, int n_matrices, int n_models, unsigned flags,
              void* stream, tl_instance** out);
int tl_destroy(tl_instance* inst);
/* Text of the last error on this instance (or of the last failed tl_create
 * when inst is NULL), copied into buf (NUL-terminated, truncated). */
int tl_last_error(const tl_instance* inst, char* buf, size_t len);
/* Device bytes this instance holds. */
int tl_device_bytes(const tl_instance* inst, size_t* out);

/* Tip data. states: [n_patterns] int8 codes, 0..S-1 observed, any other
 * value ambiguous (all-ones partial). partials: [n_patterns][S] doubles, used
 * in every category. A tip holds either states or partials. */
int tl_set_tip_states(tl_instance* inst, int tip, const int8_t* states);
int tl_set_tip_partials(tl_instance* inst, int tip, const double* partials);
/* All tips' states at once: states is [n_tips][n_patterns] int8 (row-major),
 * copied with one 2-D transfer (full speed from page-locked host memory);
 * synchronises the stream before returning. */
int tl_set_tip_states_all(tl_instance* inst, const int8_t* states);
/* Like tl_set_tip_states_all, but asynchronous and double-buffered, so the
 * upload of the next evaluation's tip states overlaps the kernels of the
 * current one: the copy runs on the instance's own copy stream into a
 * second tip-state pool (allocated on the first call), after the kernels
 * that last read that pool; the next call that launches work on the
 * instance (update_partials, root log-likelihood, pre-order, edge
 * derivatives, adjoint) makes the instance stream wait for the copy and
 * switches to that pool. states: host, [n_tips][n_patterns] int8 as for
 * tl_set_tip_states_all; it must be page-locked for the copy to be
 * asynchronous and must stay valid and unchanged until that next call's
 * work has been queued and the copy has finished (tl_sync, or the
 * instance stream, orders after it). A second call before the pool is
 * used replaces the pending upload. Errors as tl_set_tip_states_all. */
int tl_set_tip_states_all_async(tl_instance* inst, const int8_t* states);
/* Pattern weights [n_patterns] (non-negative, finite). Default 1. */
int tl_set_pattern_weights(tl_instance* inst, const double* weights);
/* Category rates rho_r [n_categories] (>= 0) and weights w_r (>= 0, summing
 * to 1 is not required). Defaults: rates 1, weights 1/R. */
int tl_set_category_rates(tl_instance* inst, const double* rates);
int tl_set_category_weights(tl_instance* inst, const double* weights);

/* Model slot set-up (Sec. "Discussion": transition matrices by numerical
 * eigendecomposition of the rate matrix, reused across patterns).
 * tl_set_model builds Q on the device for the given kind, normalises it to
 * one expected substitution per unit time, forms dQ/dtheta for every
 * parameter (normaliser included) and diagonalises the symmetrised Q by
 * FP64 Jacobi rotations. params/freqs are read as documented at TL_MODEL_*. */
int tl_set_model(tl_instance* inst, int model, int kind, const double* params,
                 int n_params, const double* freqs, int n_freqs);
/* As tl_set_model without waiting for the device: a failed device check
 * (non-positive frequency, zero mean rate, Jacobi not converged) is reported
 * by the next tl_sync or result-returning call. For use inside a stream of
 * queued work. */
int tl_set_model_async(tl_instance* inst, int model, int kind, const double* params,
                       int n_params, const double* freqs, int n_freqs);
/* A reversible rate matrix Q (row-major S x S) with stationary pi, taken as
 * given (no normalisation); diagonalised on the device. */
int tl_set_rate_matrix(tl_instance* inst, int model, const double* Q, const double* pi);
/* A host eigensystem Q = V diag(lambda) Vinv (row-major), with pi. */
int tl_set_eigen(tl_instance* inst, int model, const double* V, const double* Vinv,
                 const double* lambda, const double* pi);
/* Read back a model's FP64 Q [S*S], pi [S] and the number of dQ/dtheta
 * matrices; dq may be NULL, otherwise receives n_dq * S * S values. */
int tl_get_model(tl_instance* inst, int model, double* Q, double* pi, double* dq, int* n_dq);

/* Transition matrices (Sec. "Discussion"): for i < count,
 *   P[p_idx[i]]_r  = V diag(exp(lambda rho_r t_i)) Vinv
 *   P[dp_idx[i]]_r = V diag(rho_r lambda exp(lambda rho_r t_i)) Vinv = dP/dt
 * for every category r; dp_idx may be NULL, entries -1 are skipped.
 * edge_len must be finite and >= 0. */
int tl_update_matrices(tl_instance* inst, int model, const int* p_idx, const int* dp_idx,
                       const double* edge_len, int count);
/* Read back one matrix slot in FP64, [R][S][S]. */
int tl_get_matrix(tl_instance* inst, int mat, double* out);

/* Execute a post-order operation list. Every child must be a tip, a buffer
 * written earlier by this list, or a buffer written by an earlier call. An
 * op list may not read a buffer that it writes later, nor write a buffer
 * twice (TL_ERR_ORDER). Ops may run in any order that respects these
 * dependencies; the results do not depend on that order. */
int tl_update_partials(tl_instance* inst, const tl_op* ops, int count);

/* Post-order partials with the transition matrices formed on the fly from
 * model `model`'s eigensystem (Sec. "Discussion": with a large state space
 * and a single site pattern no matrix is reused, so P(t) is better formed
 * inside pruning). For each op, child c with edge length len_c and each
 * category r:  v_c = V (exp(lambda rho_r len_c) o (V^-1 p_c)), two S x S
 * products per pattern instead of the S^3 matrix; dest = v_1 o v_2, rescaled
 * as by tl_update_partials (the same buffers, exponents and tip rules, so
 * tl_root_loglik follows). TL_PREC_F64 instances (any S); other precisions
 * return TL_ERR_UNSUPPORTED. Ops in dependency order (TL_ERR_ORDER as for
 * tl_update_partials); the ops of one tree level share a launch. */
typedef struct {
    int dest;
    int child1;
    int child2;
    int pad;
    double len1;
    double len2;
} tl_eig_op;
int tl_update_partials_eigen(tl_instance* inst, int model, const tl_eig_op* ops, int count);

/* Root log-likelihood (Sec. "Introduction"):
 *   l_p = log(sum_r w_r sum_s pi_s root[r,p,s]) + ln2 * E_p,
 *   logL = sum_p w_p l_p   (FP64, fixed-order two-stage reduction),
 * where E_p is the root buffer's accumulated rescaling exponent and pi is the
 * model's stationary distribution. out_site_logl ([n_patterns]) may be NULL.
 * Returns TL_ERR_NUMERIC (and writes the value) when a pattern likelihood
 * is not positive and finite. */
int tl_root_loglik(tl_instance* inst, int root, int model, double* out_logl,
                   double* out_site_logl);
/* Same on the device: writes logL to out_logl_dev (1 double) without
 * synchronising; the numeric-error flag is checked by the next synchronous
 * call or tl_sync. */
int tl_root_loglik_dev(tl_instance* inst, int root, int model, double* out_logl_dev);

/* Pre-order partials (materialised in the pre[] buffers of each op). */
int tl_update_pre_partials(tl_instance* inst, const tl_pre_op* ops, int count, int model);
/* Fused pre-order pass and branch-length gradient: ops in pre-order (a
 * parent's op before its children's). q partials stay on chip where
 * possible and are written only where pre[] >= 0. out_grad has n_grad
 * doubles; slot edge[c] receives dlogL/dt_c; untouched slots are zeroed. */
int tl_pre_order_gradient(tl_instance* inst, const tl_pre_op* ops, int count, int model,
                          double* out_grad, int n_grad);
int tl_pre_order_gradient_dev(tl_instance* inst, const tl_pre_op* ops, int count, int model,
                              double* out_grad_dev, int n_grad);
/* Substitution-parameter derivative matrices (Sec. "Discussion": exact
 * gradients through the matrix exponential). For i < count and every
 * category r, slot idx[i] receives dP_r(t_i)/dtheta_param, the Frechet
 * derivative of exp(rho_r t_i Q) in the direction rho_r t_i dQ/dtheta_param,
 * computed in the eigenbasis as V [(Vinv dQ V) o Phi] Vinv with
 * Phi_jk = (e^{a_j} - e^{a_k}) / (a_j - a_k), a = rho_r t_i lambda. param
 * indexes the model's dQ/dtheta (tl_get_model reports how many). */
int tl_update_param_matrices(tl_instance* inst, int model, int param, const int* idx,
                             const double* edge_len, int count);
/* As tl_pre_order_gradient, but dmat_c may hold any derivative of P_c (for
 * example from tl_update_param_matrices): slot edge[c] receives
 *   sum_p w_p [sum_r w_r u_c^T dmat_c p_c] / [sum_r w_r u_c^T P_c p_c].
 * Summing the slots of every edge gives dlogL/dtheta. */
int tl_pre_order_derivative(tl_instance* inst, const tl_pre_op* ops, int count, int model,
                            double* out, int n_out);
/* Edge derivatives from materialised partials:
 *   g_c = sum_p w_p [sum_r w_r rho_r q_c^T Q p_c] / [sum_r w_r q_c^T p_c]. */
int tl_edge_derivatives(tl_instance* inst, const tl_edge* edges, int count, int model,
                        double* out_grad, int n_grad);

/* ---- reverse-mode adjoint ----------------------------------------------
 * One parent of tl_adjoint: its post-order buffer (parent_post), its
 * pre-order partial (parent_pre, a buffer; -1 for the root, q = pi), its two
 * children (post-order buffers or tips) with the matrix slots of their edges,
 * and for each child the output slot of its edge (edge >= 0) or -1 to leave
 * the edge out. */
typedef struct {
    int parent_post;
    int parent_pre;
    int child[2];
    int mat[2];
    int edge[2];
} tl_adj_op;

#define TL_ADJ_FIRST_ORDER 0x1u  /* dlogL/dQ by the first-order approximation
                                    dP = rho t dQ P instead of the exact
                                    adjoint (for comparison)                  */

/* Reverse-mode gradient of logL with respect to every branch length, every
 * entry of Q and every model parameter, from one pass over the stored
 * partials (Sec. "Discussion": reverse-mode gradients through the adjoint
 * of the matrix exponential; Sec. "Algorithmic advances": gradients for
 * random-effects models as dlogL/dQ times dQ/dtheta). For each listed edge
 * c (parent n, sibling s) and category r the pattern likelihood is linear in
 * P_c,r, so
 *   M_c,r = dlogL/dP_c,r = w_r sum_p (w_p / L_p) u_c[r,p] p_c[r,p]^T,
 *   u_c = q_n o (P_s p_s);
 * then, with W = V^T M_c,r V^-T and a = rho_r t_c lambda (V, lambda the
 * model's eigensystem, t_c the length the slot mat[c] was last computed with
 * by tl_update_matrices for this model):
 *   out_grad[edge]  = sum_r sum_i W_ii rho_r lambda_i exp(a_i)   (dlogL/dt_c)
 *   out_dQ          = V^-T [sum_{c,r} rho_r t_c W o Phi] V^T     (dlogL/dQ)
 *     Phi_ij = (e^{a_i} - e^{a_j}) / (a_i - a_j), e^{a_i} when a_i = a_j;
 *     with TL_ADJ_FIRST_ORDER: sum_{c,r} rho_r t_c M_c,r P_c,r^T
 *   out_dtheta[k]   = <dlogL/dQ, dQ/dtheta_k>  (k < n_theta; HKY 1, GTR 6,
 *                     GY94 2, GY94RE 265 parameters in tl_set_model order;
 *                     TL_MODEL_REV S*S, the exchangeability matrix row-major,
 *                     0 on its diagonal).
 * L_p is taken at the parent, up to the scales that cancel: from the same
 * products sum_r w_r q_n . (v_a o v_b), v_c = P_c p_c (four states), or
 * from the stored post-order partial of parent_post and its rescaling
 * exponents (any S). Inputs: post-order partials of every parent_post and
 * child, and the pre-order partials of every parent_pre
 * (tl_update_pre_partials of the same post-order partials). Root
 * frequencies are held fixed. Outputs are host
 * arrays (each may be NULL): out_grad [n_grad] (slots not listed are zeroed),
 * out_dQ [S*S] row-major, out_dtheta [n_theta] (n_theta must equal the
 * model's parameter count; models set by tl_set_rate_matrix or tl_set_eigen
 * have none). Errors: TL_ERR_STATE for a buffer or matrix slot that holds no
 * data or a slot computed for another model, TL_ERR_INDEX, TL_ERR_ARG,
 * TL_ERR_NUMERIC for a pattern with zero likelihood. */
int tl_adjoint(tl_instance* inst, const tl_adj_op* ops, int count, int model, unsigned flags,
               double* out_grad, int n_grad, double* out_dQ, double* out_dtheta, int n_theta);

/* ---- node-height ratio transform ------------------------------------------
 * Node heights and branch-specific rates inferred together through a ratio
 * transform of the node heights that keeps every node older than its
 * descendants (Sec. "Algorithmic advances"). Tree: parent[v] for the
 * 2 n_tips - 1 nodes, tips 0..n_tips-1, every internal node numbered after
 * its children (parent[v] > v), the root last with parent -1. Tip heights
 * tip_height[n_tips] are fixed; internal node n_tips + k has the ratio
 * ratio[k] in (0, 1) (the root's entry is ignored); rate[v] is the rate of
 * the branch above v (the root's ignored). With a_v the largest tip height
 * below v:
 *   h_v = a_v + r_v (h_parent(v) - a_v),   h_root = root_height,
 *   t_v = rate_v (h_parent(v) - h_v)   (expected substitutions).
 * tl_ratio_heights writes out_height and out_len ([2 n_tips - 1]; the
 * root's length 0; either may be NULL). tl_ratio_gradient takes dlogL/dt
 * (grad_len [2 n_tips - 1], e.g. from tl_pre_order_gradient) and writes, by
 * the chain rule through the transform, dlogL/dratio [n_tips - 1] (root
 * entry 0), dlogL/droot_height [1] and dlogL/drate [2 n_tips - 1] (root 0;
 * any may be NULL). Host arrays; the arithmetic runs in one device block,
 * level by level, on `stream` (a cudaStream_t or NULL), synchronously.
 * Errors (TL_ERR_ARG: malformed tree, a ratio outside (0, 1), a root height
 * not above every tip, non-finite input) are reported by
 * tl_last_error(NULL, ...). */
int tl_ratio_heights(int n_tips, const int* parent, const double* tip_height, const double* ratio,
                     double root_height, const double* rate, double* out_height,
                     double* out_len, void* stream);
int tl_ratio_gradient(int n_tips, const int* parent, const double* tip_height, const double* ratio,
                      double root_height, const double* rate, const double* grad_len,
                      double* out_grad_ratio, double* out_grad_root_height,
                      double* out_grad_rate, void* stream);

/* Read back one buffer in FP64: out [R][n_patterns][S] partials as stored
 * (post-order partials carry their accumulated power-of-two exponents
 * separately; pre-order partials are defined up to a per-pattern power of
 * two). exponents ([n_patterns] int32, may be NULL) receives the buffer's
 * accumulated rescaling exponents (zeros for pre-order buffers and tips). */
int tl_get_partials(tl_instance* inst, int buf, double* out, int32_t* exponents);

/* Root log-likelihood without any device allocation (the paper has no
 * counterpart; this exists for callers that cannot allocate device memory,
 * such as code running inside someone else's stream capture, plug-ins whose
 * host application owns the allocator, or loops that forbid allocation
 * after start-up). Computes the same value as tl_root_loglik for caller-held
 * FP32 four-state root partials:
 *   root_partials    device, [n_categories][pattern_stride][4] float, 16-byte
 *                    aligned (the layout of an FP32 instance buffer)
 *   exponents        device, [n_patterns] int32 accumulated rescaling
 *                    exponents, or NULL for none
 *   pi               device, [4] doubles; cat_weights device, [n_categories]
 *   pattern_weights  device, [n_patterns] doubles
 *   out_logl         device, 1 double, written asynchronously on `stream`
 * Scratch is a fixed array built into the library (one double per 32
 * patterns): n_patterns above 2,097,152 returns TL_ERR_UNSUPPORTED. The
 * array is a module global: the CUDA runtime loads the module that holds it
 * (and so reserves its 512 KiB) lazily, on the first use on each device,
 * not when the library is loaded. The first call on each device does that
 * set-up with the device current (it loads the module and looks up the
 * device's copy of the array, then caches the address), so make the first
 * call on each device before any stream capture. The cached address belongs
 * to the device's primary context: after cudaDeviceReset, or from another
 * context on the same device, it is no longer valid and this entry point
 * must not be used. All calls share the array, so calls that overlap on the
 * GPU (other streams, other host threads) race; serialise them. A zero or non-finite pattern
 * likelihood shows up as a non-finite *out_logl (no status is read back).
 * Errors in arguments are reported through tl_last_error(NULL, ...). */
int tl_root_loglik_static(const float* root_partials, const int32_t* exponents,
                          const double* pi, const double* cat_weights,
                          const double* pattern_weights, int n_patterns, int pattern_stride,
                          int n_categories, double* out_logl, void* stream);

/* Number of kernels this instance has launched since creation. */
int tl_launch_count(const tl_instance* inst, unsigned long long* out);

/* Wait for the instance's stream and report any pending device error. */
int tl_sync(tl_instance* inst);

/* ---- batched evaluation of several instances ------------------------------
 * Patterns are conditionally independent given the tree and so are separate
 * trees: the per-pattern updates of many instances (different trees, taxa
 * and pattern counts) are one data-parallel launch (Sec. "Benchmarks on
 * NVIDIA and AMD GPUs" splits one alignment across devices by the same
 * independence). These calls take n four-state instances (S = 4, FP32 or
 * FP64, all of one precision and category count, each at most once) and do
 * for all of them what the single-instance call does for one, with one
 * kernel launch per pass instead of one per instance. Each instance's
 * results are bit-identical to its single-instance call and do not depend on
 * the other instances in the batch.
 *
 * Streams: the batched work runs on the batch's stream, after the work
 * already queued on each instance's stream; each instance's stream then
 * waits for the batched work (events; no host synchronisation).
 * Errors: the batch's status and tl_batch_last_error; an error in instance
 * k's arguments names k and launches nothing. Output pointers are device
 * memory. */
typedef struct tl_batch tl_batch;

int tl_batch_create(void* cuda_stream, tl_batch** out);
int tl_batch_destroy(tl_batch* b);
int tl_batch_last_error(const tl_batch* b, char* buf, size_t len);
/* Kernels launched by the batch (not counted by the instances). */
int tl_batch_launch_count(const tl_batch* b, unsigned long long* out);

/* tl_update_partials for each instance k with ops[k][0 .. counts[k]). */
int tl_batch_update_partials(tl_batch* b, tl_instance* const* insts, const tl_op* const* ops,
                             const int* counts, int n);
/* tl_root_loglik_dev for each instance: out_logl_dev[k] (device, n doubles)
 * receives logL of instance k at buffer roots[k] under model models[k]. */
int tl_batch_root_loglik_dev(tl_batch* b, tl_instance* const* insts, const int* roots,
                             const int* models, int n, double* out_logl_dev);
/* tl_pre_order_gradient_dev for each instance: out_grad_dev[k] (device,
 * n_grad[k] doubles) receives instance k's branch-length gradient. */
int tl_batch_pre_order_gradient_dev(tl_batch* b, tl_instance* const* insts,
                                    const tl_pre_op* const* ops, const int* counts,
                                    const int* models, double* const* out_grad_dev,
                                    const int* n_grad, int n);

#ifdef __cplusplus
}
#endif
#endif /* TREELIK_H */
