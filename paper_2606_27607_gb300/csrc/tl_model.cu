// Rate matrices, their FP64 eigensystems and the transition matrices.
//
// The paper computes transition probability matrices from a numerical
// eigendecomposition of the instantaneous rate matrix and caches them for
// reuse across site patterns (Sec. "Discussion"). Here every step runs on the
// device in FP64: Q is built from the model parameters and normalised to one
// expected substitution per unit time, the reversible Q is symmetrised as
// D^1/2 Q D^-1/2 (D = diag(pi)) and diagonalised by cyclic Jacobi rotations
// in a round-robin (tournament) order, and P_r(t) = V diag(exp(lambda rho_r t))
// Vinv and dP_r/dt = V diag(rho_r lambda exp(lambda rho_r t)) Vinv are formed
// per edge and category. Working-precision copies are laid out for the
// kernels that consume them.
#include <cmath>

#include <type_traits>

#include "tl_df.cuh"
#include "tl_internal.cuh"

namespace tl {

// Standard genetic code, first/second/third base in A,C,G,T order; '*' marks
// the stop codons.
__constant__ char c_code_acgt[65] =
    "KNKNTTTTRSRSIIMIQHQHPPPPRRRRLLLLEDEDAAAAGGGGVVVV*Y*YSSSS*CWCLFLF";

__device__ __forceinline__ bool is_transition(int x, int y) {
    return (x == 0 && y == 2) || (x == 2 && y == 0) || (x == 1 && y == 3) || (x == 3 && y == 1);
}

// Build Q, pi and dQ/dtheta for one model slot. One block.
__device__ __forceinline__ bool one_difference(int ci, int cj) {
    const int x = ci ^ cj;  // two bits per position
    return ((x & 0x30) != 0) + ((x & 0x0c) != 0) + ((x & 0x03) != 0) == 1;
}

// Build Q, pi and dQ/dtheta for one model slot. One block. Random-effects
// GY94 numbers the unordered one-difference pairs (i < j) lexicographically
// (row counts, a prefix sum, then each row's pairs) and writes that list.
__global__ void k_build_model(int kind, int S, int Spad, const double* __restrict__ params,
                              const double* __restrict__ freqs, double* __restrict__ Q,
                              double* __restrict__ pi, double* __restrict__ dQ, int n_dq,
                              int* __restrict__ pairs, double* __restrict__ mu_out,
                              int* __restrict__ err) {
    __shared__ int codon_nt[64];   // sense codon -> 16*n1 + 4*n2 + n3
    __shared__ char codon_aa[64];
    __shared__ short pair_of[61 * 61];  // random effects: pair index of (i, j), i < j
    __shared__ int row_start[62];
    __shared__ double s_pi[64];
    __shared__ double s_red[256];
    __shared__ double s_mu[1 + kMaxDq];
    __shared__ double s_q[64 * 64];   // off-diagonal rates (S <= 64)
    const int t = threadIdx.x;
    const int nt = blockDim.x;

    if (t == 0) {
        int k = 0;
        for (int c = 0; c < 64; ++c) {
            if (c_code_acgt[c] == '*') continue;
            codon_nt[k] = c;
            codon_aa[k] = c_code_acgt[c];
            ++k;
        }
    }
    __syncthreads();
    const bool codon = kind == TL_MODEL_GY94 || kind == TL_MODEL_GY94RE;
    if (kind == TL_MODEL_GY94RE) {
        if (t < 61) {
            int n = 0;
            for (int j = t + 1; j < 61; ++j) n += one_difference(codon_nt[t], codon_nt[j]);
            row_start[t + 1] = n;
        }
        __syncthreads();
        if (t == 0) {
            row_start[0] = 0;
            for (int i = 1; i <= 61; ++i) row_start[i] += row_start[i - 1];
        }
        __syncthreads();
        if (t < 61) {
            int k = row_start[t];
            for (int j = t + 1; j < 61; ++j)
                if (one_difference(codon_nt[t], codon_nt[j])) {
                    pair_of[t * 61 + j] = (short)k;
                    pairs[2 * k] = t;
                    pairs[2 * k + 1] = j;
                    ++k;
                }
        }
        __syncthreads();
    }
    // stationary frequencies
    if (codon) {
        for (int i = t; i < 61; i += nt) {
            int c = codon_nt[i];
            s_pi[i] = freqs[c >> 4] * freqs[4 + ((c >> 2) & 3)] * freqs[8 + (c & 3)];
        }
        __syncthreads();
        if (t == 0) {
            double z = 0;
            for (int i = 0; i < 61; ++i) z += s_pi[i];
            for (int i = 0; i < 61; ++i) s_pi[i] /= z;
        }
    } else {
        for (int i = t; i < S; i += nt) s_pi[i] = freqs[i];
    }
    __syncthreads();
    for (int i = t; i < Spad; i += nt) pi[i] = i < S ? s_pi[i] : 0.0;

    // off-diagonal rates R_ij = s_ij pi_j and their parameter derivatives
    for (int idx = t; idx < Spad * Spad; idx += nt) {
        int i = idx / Spad, j = idx % Spad;
        double r = 0.0;
        double d[kMaxDq];
        for (int k = 0; k < kMaxDq; ++k) d[k] = 0.0;
        if (i < S && j < S && i != j) {
            if (kind == TL_MODEL_HKY) {
                bool ts = is_transition(i, j);
                r = (ts ? params[0] : 1.0) * s_pi[j];
                d[0] = ts ? s_pi[j] : 0.0;
            } else if (kind == TL_MODEL_GTR) {
                int a = min(i, j), b = max(i, j);
                // pair order AC AG AT CG CT GT
                int k = (a == 0) ? (b - 1) : (a == 1 ? (b + 1) : 5);
                r = params[k] * s_pi[j];
                d[k] = s_pi[j];
            } else if (codon) {
                int ci = codon_nt[i], cj = codon_nt[j];
                int ndiff = 0, pos = -1;
                for (int q = 0; q < 3; ++q) {
                    int sh = 4 - 2 * q;
                    if (((ci >> sh) & 3) != ((cj >> sh) & 3)) {
                        ++ndiff;
                        pos = sh;
                    }
                }
                if (ndiff == 1) {
                    bool ts = is_transition((ci >> pos) & 3, (cj >> pos) & 3);
                    bool ns = codon_aa[i] != codon_aa[j];
                    double kap = ts ? params[0] : 1.0;
                    double om = ns ? params[1] : 1.0;
                    const double m = (kind == TL_MODEL_GY94RE)
                                         ? exp(params[2 + pair_of[min(i, j) * 61 + max(i, j)]])
                                         : 1.0;
                    r = kap * om * s_pi[j] * m;
                    d[0] = (ts ? 1.0 : 0.0) * om * s_pi[j] * m;
                    d[1] = kap * (ns ? 1.0 : 0.0) * s_pi[j] * m;
                }
            } else {  // TL_MODEL_REV
                r = 0.5 * (params[i * S + j] + params[j * S + i]) * s_pi[j];
            }
        }
        Q[idx] = r;
        if (i < S && j < 64) s_q[i * 64 + j] = r;
        for (int k = 0; k < n_dq; ++k) dQ[(size_t)k * Spad * Spad + idx] = d[k];
    }
    __syncthreads();
    // diagonals (row sums) of R (from the shared copy) and of each dR
    for (int i = t; i < S; i += nt) {
        double acc = 0;
        for (int j = 0; j < S; ++j)
            if (j != i) acc += s_q[i * 64 + j];
        Q[i * Spad + i] = -acc;
        for (int k = 0; k < n_dq; ++k) {
            double* D = dQ + (size_t)k * Spad * Spad;
            double a2 = 0;
            for (int j = 0; j < S; ++j)
                if (j != i) a2 += D[i * Spad + j];
            D[i * Spad + i] = -a2;
        }
    }
    __syncthreads();
    // normalisers mu = -sum pi_i R_ii and dmu_k
    for (int k = 0; k <= n_dq; ++k) {
        const double* M = (k == 0) ? Q : dQ + (size_t)(k - 1) * Spad * Spad;
        double acc = 0;
        for (int i = t; i < S; i += nt) acc -= s_pi[i] * M[i * Spad + i];
        s_red[t] = acc;
        __syncthreads();
        for (int w = nt / 2; w > 0; w >>= 1) {
            if (t < w) s_red[t] += s_red[t + w];
            __syncthreads();
        }
        if (t == 0) s_mu[k] = s_red[0];
        __syncthreads();
    }
    const double mu = s_mu[0];
    if (t == 0 && !(mu > 0.0 && isfinite(mu))) err[0] = 1;
    if (t == 0) mu_out[0] = mu;
    // Q / mu exactly; the derivatives (which only feed parameter gradients)
    // through one reciprocal, not a division per element and parameter
    const double inv_mu = 1.0 / mu, inv_mu2 = inv_mu * inv_mu;
    for (int idx = t; idx < Spad * Spad; idx += nt) {
        double r = Q[idx];
        for (int k = 0; k < n_dq; ++k) {
            double* D = dQ + (size_t)k * Spad * Spad;
            D[idx] = D[idx] * inv_mu - r * s_mu[k + 1] * inv_mu2;
        }
        Q[idx] = r / mu;
    }
}

// off(A)^2 and diag(A)^2 of the n x n block A (leading dimension LD), summed
// in FP64 (a tree over the block's threads); every thread gets both.
template <typename T>
__device__ void off_diag_sums(const T* A, int n, int LD, double* s_red, double& offs,
                              double& dgs) {
    const int t = threadIdx.x, nt = blockDim.x;
    double off = 0, dg = 0;
    for (int idx = t; idx < n * n; idx += nt) {
        int i = idx / n, j = idx % n;
        double a = (double)A[i * LD + j];
        if (i == j) dg += a * a;
        else off += a * a;
    }
    s_red[t] = off;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
        if (t < w) s_red[t] += s_red[t + w];
        __syncthreads();
    }
    offs = s_red[0];
    __syncthreads();
    s_red[t] = dg;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
        if (t < w) s_red[t] += s_red[t + w];
        __syncthreads();
    }
    dgs = s_red[0];
    __syncthreads();
}

// One block-wide sweep set of cyclic Jacobi in tournament order on the
// symmetric n x n matrix A (leading dimension LD), accumulating the
// rotations into the columns of U. Each round rotates m / 2 disjoint pairs
// at once. Stops after `settle` sweeps have ended with off(A)^2 <= done_tol *
// diag(A)^2, once a sweep near the diagonal (off(A)^2 <= 1e-8 diag(A)^2)
// leaves off(A)^2 above stall * its previous value (stall > 0: the rounding
// floor of T is reached), or after max_sweeps;
// returns (to every thread) whether off(A)^2 <= conv_tol * diag(A)^2 at the
// end.
template <typename T>
__device__ bool jacobi_sweeps(T* A, T* U, int n, int LD, int max_sweeps, double done_tol,
                              double conv_tol, int settle, double stall, T* s_c, T* s_s,
                              int* s_p, int* s_q, double* s_red, int* s_flag) {
    const int t = threadIdx.x, nt = blockDim.x;
    const int warp_id = t >> 5, ln = t & 31, n_warps = nt >> 5;
    const int m = (n + 1) & ~1;  // players in the tournament (one dummy if n odd)
    int done = 0;
    bool conv = false;
    double prev = -1.0;  // off(A)^2 after the previous sweep (thread 0)
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int round = 0; round < m - 1; ++round) {
            if (t < m / 2) {
                int a = t, b = m - 1 - t;
                int pa = (a == 0) ? 0 : ((a - 1 + round) % (m - 1)) + 1;
                int pb = (b == 0) ? 0 : ((b - 1 + round) % (m - 1)) + 1;
                int p = min(pa, pb), q = max(pa, pb);
                T c = T(1), sn = T(0);
                if (q < n) {
                    T apq = A[p * LD + q];
                    if (fabs((double)apq) > 1e-300) {
                        T theta = (A[q * LD + q] - A[p * LD + p]) / (T(2) * apq);
                        T tt = T(1) / (fabs(theta) + sqrt(theta * theta + T(1)));
                        if (theta < 0) tt = -tt;
                        c = T(1) / sqrt(tt * tt + T(1));
                        sn = tt * c;
                    }
                } else {
                    p = q = -1;
                }
                s_c[t] = c;
                s_s[t] = sn;
                s_p[t] = p;
                s_q[t] = q;
            }
            __syncthreads();
            // rows: A <- J^T A (a warp per rotation, a lane per column)
            for (int k = warp_id; k < m / 2; k += n_warps) {
                const int p = s_p[k], q = s_q[k];
                if (p < 0 || s_s[k] == T(0)) continue;
                const T c = s_c[k], sn = s_s[k];
                for (int j = ln; j < n; j += 32) {
                    const T ap = A[p * LD + j], aq = A[q * LD + j];
                    A[p * LD + j] = c * ap - sn * aq;
                    A[q * LD + j] = sn * ap + c * aq;
                }
            }
            __syncthreads();
            // columns: A <- A J, U <- U J (a warp per rotation, a lane per row)
            for (int k = warp_id; k < m / 2; k += n_warps) {
                const int p = s_p[k], q = s_q[k];
                if (p < 0 || s_s[k] == T(0)) continue;
                const T c = s_c[k], sn = s_s[k];
                for (int i = ln; i < n; i += 32) {
                    const T ap = A[i * LD + p], aq = A[i * LD + q];
                    A[i * LD + p] = c * ap - sn * aq;
                    A[i * LD + q] = sn * ap + c * aq;
                    const T up = U[i * LD + p], uq = U[i * LD + q];
                    U[i * LD + p] = c * up - sn * uq;
                    U[i * LD + q] = sn * up + c * uq;
                }
            }
            __syncthreads();
        }
        // convergence: off-diagonal mass relative to the diagonal
        double offs, dgs;
        off_diag_sums(A, n, LD, s_red, offs, dgs);
        if (t == 0) {
            s_flag[0] = offs <= done_tol * dgs;
            s_flag[1] = offs <= conv_tol * dgs;
            // stalled: within 1e-8 of the diagonal and no longer shrinking fast
            s_flag[2] = stall > 0.0 && prev >= 0.0 && offs > stall * prev &&
                        offs <= 1e-8 * dgs;
            prev = offs;
        }
        __syncthreads();
        done += s_flag[0];
        conv = s_flag[1];
        const bool stalled = s_flag[2];
        __syncthreads();
        if (done >= settle || stalled) break;
    }
    return conv;
}

// C = A^T B (transA) or A B for n x n blocks in shared memory (leading
// dimension LD), FP64.
__device__ void smem_gemm64(const double* A, const double* B, double* C, int n, int LD,
                            bool transA) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx / n, j = idx % n;
        double acc = 0.0;
        for (int k = 0; k < n; ++k)
            acc += (transA ? A[k * LD + i] : A[i * LD + k]) * B[k * LD + j];
        C[i * LD + j] = acc;
    }
    __syncthreads();
}

// The same products on many SMs, a block per row of Z (a thread per column):
// Z = X Y or X^T Y (row stride LD), or with ns the Newton-Schulz factor
// (3 I - X^T Y) / 2; each element summed as in smem_gemm64.
__global__ void __launch_bounds__(64) k_eig_gemm(int n, int LD, const double* __restrict__ X,
                                                 const double* __restrict__ Y,
                                                 double* __restrict__ Z, int transX, int ns) {
    const int i = blockIdx.x, j = threadIdx.x;
    if (j >= n) return;
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc += (transX ? X[k * LD + i] : X[i * LD + k]) * Y[k * LD + j];
    Z[i * LD + j] = ns ? 0.5 * ((i == j ? 3.0 : 0.0) - acc) : acc;
}

// Largest rotation sine a simultaneous refinement step takes; a pair whose
// rotation is larger (eigenvalues close on the scale of their coupling) is
// left to the Jacobi sweeps that follow.
constexpr double kRefineMaxSine = 1e-3;

// All the Jacobi rotations of a nearly diagonal symmetric A at once:
// G = I + Theta with Theta antisymmetric, Theta_pq = s_pq (p < q) the sine
// of the plane rotation that zeroes A_pq, signed as the rotations of
// jacobi_sweeps (U <- U J, J_pq = s, J_qp = -s). To first order G^T A G
// has no off-diagonal part; the second-order remainder is about
// off(A)^2 / gap, so each step squares the relative off-diagonal size
// (a block per row, a thread per column).
__global__ void __launch_bounds__(64) k_eig_rot(int n, int LD, const double* __restrict__ A,
                                                double* __restrict__ G) {
    const int i = blockIdx.x, j = threadIdx.x;
    if (j >= n) return;
    double g = 1.0;
    if (i != j) {
        const int p = min(i, j), q = max(i, j);
        const double apq = 0.5 * (A[p * LD + q] + A[q * LD + p]);
        double s = 0.0;
        if (fabs(apq) > 1e-300) {
            const double theta = (A[q * LD + q] - A[p * LD + p]) / (2.0 * apq);
            double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
            if (theta < 0) t = -t;
            s = t / sqrt(t * t + 1.0);
            if (fabs(s) > kRefineMaxSine) s = 0.0;
        }
        g = (i == p) ? s : -s;
    }
    G[i * LD + j] = g;
}

// Threads of the eigensolver's block: 256 for up to 32 states; above that
// 1,024, so that a Jacobi round's rotations (up to 32) each get a warp and
// the block-wide passes over the matrix have four times the threads.
constexpr int kEigThreadsMax = 1024;

// Eigensystem of the reversible Q through the symmetric form
// A = D^1/2 Q D^-1/2 (D = diag(pi)), A = U diag(lambda) U^T, so
// V = D^-1/2 U and Vinv = U^T D^1/2. One block, in two precisions: cyclic
// Jacobi in FP32 brings A near diagonal at FP32 cost (FP64 issue is far
// slower on this part); the FP32 rotations U32 are then made orthogonal to
// FP64 accuracy by two Newton-Schulz steps U <- U (3 I - U^T U) / 2, A is
// transformed to U^T A U in FP64, and FP64 Jacobi sweeps (accumulated onto
// U) finish it, converging quadratically from the FP32 starting point.
//
// phase 0 runs all of it in the one block; for large S the FP64 products run
// on many SMs instead: phase 1 stops after the FP32 sweeps and writes A and
// U (row stride Spad) to scratch[0] and scratch[1]; k_eig_gemm forms the
// Newton-Schulz steps and U^T A U (each element summed in the same order as
// here, so the result is the same) and two simultaneous-rotation steps
// (k_eig_rot) refine U and U^T A U; phase 2 reads U from scratch[1] and
// U^T A U from scratch[3] and runs the FP64 sweeps only if the off-diagonal
// part is still above their stopping threshold (eigenvalues too close for
// the refinement).
__global__ void __launch_bounds__(kEigThreadsMax) k_eigen(int S, int Spad, const double* __restrict__ Q,
                        const double* __restrict__ pi, double* __restrict__ V,
                        double* __restrict__ Vinv, double* __restrict__ lam,
                        int* __restrict__ err, int phase, double* __restrict__ scratch) {
    extern __shared__ double sm[];
    constexpr int LD = 65;
    double* A = sm;                   // [64][LD] FP64
    double* U = A + 64 * LD;          // [64][LD]
    double* T1 = U + 64 * LD;         // [64][LD] scratch
    double* T2 = T1 + 64 * LD;        // [64][LD] scratch
    float* A32 = reinterpret_cast<float*>(T2 + 64 * LD);   // [64][LD]
    float* U32 = A32 + 64 * LD;                            // [64][LD]
    __shared__ double s_sq[64], s_isq[64];   // sqrt(pi_i) and its reciprocal
    __shared__ double s_c[32], s_s[32];
    __shared__ float s_cf[32], s_sf[32];
    __shared__ int s_p[32], s_q[32];
    __shared__ double s_red[kEigThreadsMax];
    __shared__ int s_flag[3];
    const int t = threadIdx.x, nt = blockDim.x;
    const int n = S;

    for (int i = t; i < n; i += nt) {
        double p = pi[i];
        s_sq[i] = sqrt(p);
        s_isq[i] = 1.0 / s_sq[i];
        if (!(p > 0.0)) err[0] = 2;
    }
    __syncthreads();
    if (phase == 2) {
        const size_t SS = (size_t)Spad * Spad;
        for (int idx = t; idx < n * n; idx += nt) {
            const int i = idx / n, j = idx % n;
            U[i * LD + j] = scratch[SS + i * Spad + j];
            A[i * LD + j] = 0.5 * (scratch[3 * SS + i * Spad + j] + scratch[3 * SS + j * Spad + i]);
        }
        __syncthreads();
    } else {
    for (int idx = t; idx < n * n; idx += nt) {
        int i = idx / n, j = idx % n;
        // symmetrise: (D^1/2 Q D^-1/2 + transpose) / 2
        double a = s_sq[i] * Q[i * Spad + j] * s_isq[j];
        double b = s_sq[j] * Q[j * Spad + i] * s_isq[i];
        const double v = 0.5 * (a + b);
        A[i * LD + j] = v;
        A32[i * LD + j] = (float)v;
        U32[i * LD + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    // FP32: until off(A)^2 <= 1e-12 diag(A)^2 (about FP32 rounding), 20 sweeps at most
    jacobi_sweeps<float>(A32, U32, n, LD, 20, 1e-12, 1e-12, 1, 0.1, s_cf, s_sf, s_p, s_q, s_red,
                         s_flag);
    // FP64 orthonormalisation of the FP32 rotations
    for (int idx = t; idx < n * n; idx += nt) {
        const int i = idx / n, j = idx % n;
        U[i * LD + j] = (double)U32[i * LD + j];
    }
    __syncthreads();
    if (phase == 1) {
        const size_t SS = (size_t)Spad * Spad;
        for (int idx = t; idx < n * n; idx += nt) {
            const int i = idx / n, j = idx % n;
            scratch[i * Spad + j] = A[i * LD + j];
            scratch[SS + i * Spad + j] = U[i * LD + j];
        }
        return;
    }
    for (int it = 0; it < 2; ++it) {
        smem_gemm64(U, U, T1, n, LD, true);          // T1 = U^T U
        for (int idx = t; idx < n * n; idx += nt) {
            const int i = idx / n, j = idx % n;
            T1[i * LD + j] = 0.5 * ((i == j ? 3.0 : 0.0) - T1[i * LD + j]);
        }
        __syncthreads();
        smem_gemm64(U, T1, T2, n, LD, false);        // T2 = U (3 I - U^T U) / 2
        for (int idx = t; idx < n * n; idx += nt) {
            const int i = idx / n, j = idx % n;
            U[i * LD + j] = T2[i * LD + j];
        }
        __syncthreads();
    }
    // A <- U^T A U in FP64, symmetrised
    smem_gemm64(A, U, T1, n, LD, false);             // T1 = A U
    smem_gemm64(U, T1, T2, n, LD, true);             // T2 = U^T A U
    for (int idx = t; idx < n * n; idx += nt) {
        const int i = idx / n, j = idx % n;
        A[i * LD + j] = 0.5 * (T2[i * LD + j] + T2[j * LD + i]);
    }
    __syncthreads();
    }
    // FP64: stop once off(A)^2 <= 1e-28 diag(A)^2 (off-diagonal at 1e-14 of
    // the diagonal; from the FP32 start one or two sweeps); fail above 1e-24
    // (phase 2: the refinement steps before it usually leave A below that
    // already, and then no sweep runs)
    double offs = 1.0, dgs = 0.0;
    if (phase == 2) off_diag_sums(A, n, LD, s_red, offs, dgs);
    const bool conv = (phase == 2 && offs <= 1e-28 * dgs) ||
                      jacobi_sweeps<double>(A, U, n, LD, 40, 1e-28, 1e-24, 1, 0.0, s_c, s_s, s_p,
                                            s_q, s_red, s_flag);
    if (t == 0 && !conv) err[0] = 3;
    for (int idx = t; idx < Spad * Spad; idx += nt) {
        int i = idx / Spad, k = idx % Spad;
        double v = 0, vi = 0;
        if (i < n && k < n) {
            v = U[i * LD + k] * s_isq[i];   // V = D^-1/2 U
            vi = U[k * LD + i] * s_sq[k];  // Vinv[i][k] = U[k][i] sqrt(pi_k)
        }
        V[idx] = v;
        Vinv[idx] = vi;
    }
    for (int i = t; i < Spad; i += nt) lam[i] = (i < n) ? A[i * LD + i] : 0.0;
}

__device__ __forceinline__ float round_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// The TF32 value of x with the low 13 mantissa bits cleared (toward zero).
__device__ __forceinline__ float trunc_tf32(float x) {
    return __uint_as_float(__float_as_uint(x) & 0xffffe000u);
}

// Double-float copies of V and Vinv for the reduced-precision matrix
// products (k_tpm).
__global__ void k_df_pairs(int n, const double* __restrict__ V, const double* __restrict__ Vinv,
                           df2* __restrict__ Vdf, df2* __restrict__ Vinvdf) {
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        Vdf[idx] = df_of(V[idx]);
        Vinvdf[idx] = df_of(Vinv[idx]);
    }
}

// Working-precision copies of pi and Q.
template <typename T>
__global__ void k_model_working(int S, int Spad, const double* __restrict__ Q,
                                const double* __restrict__ pi, T* __restrict__ Qw,
                                T* __restrict__ piw, int tf32) {
    for (int idx = threadIdx.x; idx < Spad * Spad; idx += blockDim.x) {
        T v = (T)Q[idx];
        Qw[idx] = v;
    }
    for (int i = threadIdx.x; i < Spad; i += blockDim.x) piw[i] = (T)pi[i];
    (void)S;
    (void)tf32;
}

// Write one category of one matrix slot (Pm, FP64 [Spad][Spad] in shared
// memory) into the working layout of the instance.
template <typename T>
__device__ void write_layout(const double* Pm, int slot, int r, int S, int Spad, int R,
                             T* __restrict__ matw, size_t matw_stride, int layout,
                             T* __restrict__ rowsum) {
    const int t = threadIdx.x, nt = blockDim.x;
    T* w = matw + (size_t)slot * matw_stride;
    if (layout == 0) {
        // [5 columns][R][4]: column j of every category contiguous; the
        // row-sum column (ambiguous tips) is summed in T in column order,
        // exactly as a product with an all-ones partial rounds
        for (int idx = t; idx < kColStride * 4; idx += nt) {
            int j = idx / 4, i = idx % 4;
            T v;
            if (j < 4) {
                v = (T)Pm[i * Spad + j];
            } else {
                v = (T)Pm[i * Spad];
                for (int q = 1; q < S; ++q) v = v + (T)Pm[i * Spad + q];
            }
            w[((size_t)j * R + r) * 4 + i] = v;
        }
    } else if (layout == 1) {
        w += (size_t)r * (Spad + 1) * Spad;
        for (int idx = t; idx < (Spad + 1) * Spad; idx += nt) {
            int j = idx / Spad, i = idx % Spad;
            T v;
            if (j < Spad) {
                v = (T)Pm[i * Spad + j];
            } else {
                v = (T)Pm[i * Spad];
                for (int q = 1; q < S; ++q) v = v + (T)Pm[i * Spad + q];
            }
            w[idx] = v;
        }
    } else if (layout == 2) {
        // tensor-core layout [2][R][64][64]: P row-major (the B operand)
        // and P^T (tip lookups), both TF32-rounded; row sums of the
        // rounded P summed in order (ambiguous tips)
        T* wp = w + (size_t)r * Spad * Spad;
        T* wt = w + ((size_t)R + r) * Spad * Spad;
        for (int idx = t; idx < Spad * Spad; idx += nt) {
            const int i = idx / Spad, j = idx % Spad;
            const T v = (T)round_tf32((float)Pm[idx]);
            wp[idx] = v;
            wt[j * Spad + i] = v;
        }
        __syncthreads();
        for (int i = t; i < Spad; i += nt) {
            T v = wp[i * Spad];
            for (int q = 1; q < S; ++q) v = v + wp[i * Spad + q];
            rowsum[((size_t)slot * R + r) * Spad + i] = v;
        }
    } else {
        // split tensor-core layout [4][R][64][64]: P_hi, P_hi^T, P_lo,
        // P_lo^T with P_hi = TF32(P) (nearest) and P_lo = the TF32
        // truncation of fl32(P) - P_hi. P_hi + P_lo is then exact in FP32
        // (its bits lie within those of fl32(P), or of P_hi when it rounded
        // up to the next binade), so a product with a one-hot partial, hi
        // term then lo term, gives the same FP32 value as adding the two
        // looked-up entries. Row sums of P_hi + P_lo in order.
        T* wp = w + (size_t)r * Spad * Spad;
        T* wt = w + ((size_t)R + r) * Spad * Spad;
        T* lp = w + ((size_t)2 * R + r) * Spad * Spad;
        T* lt = w + ((size_t)3 * R + r) * Spad * Spad;
        for (int idx = t; idx < Spad * Spad; idx += nt) {
            const int i = idx / Spad, j = idx % Spad;
            const float f = (float)Pm[idx];
            const float hi = round_tf32(f);
            const float lo = trunc_tf32(f - hi);
            wp[idx] = (T)hi;
            wt[j * Spad + i] = (T)hi;
            lp[idx] = (T)lo;
            lt[j * Spad + i] = (T)lo;
        }
        __syncthreads();
        for (int i = t; i < Spad; i += nt) {
            T v = wp[i * Spad] + lp[i * Spad];
            for (int q = 1; q < S; ++q) v = v + (wp[i * Spad + q] + lp[i * Spad + q]);
            rowsum[((size_t)slot * R + r) * Spad + i] = v;
        }
    }

}

// write_layout for the TF32 layouts (2, 3) from FP32 values in shared
// memory (the double-float sums rounded to FP32); the row sums are formed
// from the same rounded values, in the same order, as write_layout's. The
// transposed copies go through a padded shared-memory tile (tr, Spad rows
// of Spad + 1 floats, which fits the Spad x Spad doubles it reuses) so
// that every global store is coalesced.
template <typename T>
__device__ void write_layout_f(const float* Pf, int slot, int r, int S, int Spad, int R,
                               T* __restrict__ matw, size_t matw_stride, int layout,
                               T* __restrict__ rowsum, float* tr) {
    const int t = threadIdx.x, nt = blockDim.x;
    const int TLD = Spad + 1;
    T* w = matw + (size_t)slot * matw_stride;
    for (int part = 0; part < (layout == 3 ? 2 : 1); ++part) {   // P_hi, then P_lo
        T* wp = w + ((size_t)2 * part * R + r) * Spad * Spad;
        T* wt = w + ((size_t)(2 * part + 1) * R + r) * Spad * Spad;
        for (int idx = t; idx < Spad * Spad; idx += nt) {
            const int i = idx / Spad, j = idx % Spad;
            const float f = Pf[idx];
            const float hi = round_tf32(f);
            const float v = part == 0 ? hi : trunc_tf32(f - hi);
            wp[idx] = (T)v;
            tr[i * TLD + j] = v;
        }
        __syncthreads();
        for (int idx = t; idx < Spad * Spad; idx += nt) {
            const int j = idx / Spad, i = idx % Spad;
            wt[idx] = (T)tr[i * TLD + j];
        }
        __syncthreads();
    }
    for (int i = t; i < Spad; i += nt) {
        T v;
        if (layout == 3) {
            const float f0 = Pf[i * Spad], h0 = round_tf32(f0);
            v = (T)h0 + (T)trunc_tf32(f0 - h0);
            for (int q = 1; q < S; ++q) {
                const float f = Pf[i * Spad + q], h = round_tf32(f);
                v = v + ((T)h + (T)trunc_tf32(f - h));
            }
        } else {
            v = (T)round_tf32(Pf[i * Spad]);
            for (int q = 1; q < S; ++q) v = v + (T)round_tf32(Pf[i * Spad + q]);
        }
        rowsum[((size_t)slot * R + r) * Spad + i] = v;
    }
}

// P and dP/dt for `count` edges; grid (count, R).
//  layout 0: four-state column layout [R][5][4] of T: column j of P, then row sums
//  layout 1: FP64 transposed layout [R][Spad+1][Spad]: W[j][i] = P[i][j], row Spad = row sums
//  layout 2: TF32 row-major [R][Spad][Spad] floats (rounded) + row sums [R][Spad]
//  layout 3: layout 2 as hi and lo TF32 terms (TL_SPLIT_MATRICES)
// The TF32 layouts take the S^3 product in double-float arithmetic on the
// FP32 cores (about 2^-48 of the sum of the terms' magnitudes, far inside
// what TF32 hi + lo storage keeps; FP64 issue was this kernel's limit),
// from the model's double-float copies of V and Vinv (Vdf, Vinvdf) and
// W = V diag(e) formed as double-float products; the FP64 matrix each
// writes is that sum rounded to FP64, the working copy its FP32 rounding.
template <typename T>
__global__ void k_tpm(int S, int Spad, int R, const double* __restrict__ V,
                      const double* __restrict__ Vinv, const df2* __restrict__ Vdf,
                      const df2* __restrict__ Vinvdf, const double* __restrict__ lam,
                      const int* __restrict__ pidx, const int* __restrict__ dpidx,
                      const double* __restrict__ len, const double* __restrict__ rates,
                      double* __restrict__ mat64, T* __restrict__ matw, size_t matw_stride,
                      int layout, T* __restrict__ rowsum) {
    extern __shared__ double sm_tpm[];
    double* e = sm_tpm;              // [Spad]
    double* de = sm_tpm + 64;        // [Spad]
    double* Pm = sm_tpm + 128;       // [Spad*Spad] this matrix (for working copies)
    double* Vi = Pm + Spad * Spad;   // [Spad*Spad] Vinv
    double* W = Vi + Spad * Spad;    // [Spad*Spad] V diag(e) of the current pass
    const int b = blockIdx.x, r = blockIdx.y;
    const int t = threadIdx.x, nt = blockDim.x;
    const double rt = rates[r] * len[b];
    // P = I + V diag(expm1(lambda rho t)) Vinv keeps short branches accurate
    // (the eigen sum then carries only the O(t) part); dP/dt has no identity.
    for (int k = t; k < Spad; k += nt) {
        e[k] = (k < S) ? expm1(lam[k] * rt) : 0.0;
        de[k] = (k < S) ? rates[r] * lam[k] * exp(lam[k] * rt) : 0.0;
    }
    const bool dfp = std::is_same<T, float>::value && layout >= 2;
    df2* Vid = reinterpret_cast<df2*>(Vi);   // the same storage, as hi + lo pairs
    df2* Wd = reinterpret_cast<df2*>(W);
    float* Pf = reinterpret_cast<float*>(Pm);   // dfp: the FP32 working values
    __shared__ df2 evd[64];
    for (int idx = t; idx < Spad * Spad; idx += nt) {
        if (dfp) Vid[idx] = Vinvdf[idx];
        else Vi[idx] = Vinv[idx];
    }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        const int slot = (pass == 0) ? pidx[b] : (dpidx ? dpidx[b] : -1);
        if (slot < 0) continue;
        const double* ev = (pass == 0) ? e : de;
        // W = V diag(ev): FP64, rounded as the product V_ik ev_k was before
        // each term's fused multiply-add; double-float products for dfp
        if (dfp) {
            for (int k = t; k < Spad; k += nt) evd[k] = df_of(ev[k]);
            __syncthreads();
            for (int idx = t; idx < Spad * Spad; idx += nt) Wd[idx] = df_mul(Vdf[idx], evd[idx % Spad]);
        } else {
            for (int idx = t; idx < Spad * Spad; idx += nt) W[idx] = V[idx] * ev[idx % Spad];
        }
        __syncthreads();
        double* out = mat64 + ((size_t)slot * R + r) * Spad * Spad;
        for (int idx = t; idx < Spad * Spad; idx += nt) {
            int i = idx / Spad, j = idx % Spad;
            double acc = 0.0;
            if (dfp) {
                float f = 0.f;
                if (i < S && j < S) {
                    float sh = 0.f, sc = 0.f;
                    for (int k = 0; k < S; ++k) df_mac(sh, sc, Wd[i * Spad + k], Vid[k * Spad + j]);
                    const df2 d = df_norm(sh, sc);
                    acc = (double)d.hi + (double)d.lo;
                    f = d.hi;
                }
                if (pass == 0 && i == j && i < S) {
                    acc += 1.0;
                    f = (float)acc;
                }
                out[idx] = acc;
                Pf[idx] = f;
                continue;
            }
            if (i < S && j < S)
                for (int k = 0; k < S; ++k) acc += W[i * Spad + k] * Vi[k * Spad + j];
            if (pass == 0 && i == j && i < S) acc += 1.0;
            out[idx] = acc;
            Pm[idx] = acc;
        }
        __syncthreads();
        if (dfp)
            write_layout_f(Pf, slot, r, S, Spad, R, matw, matw_stride, layout, rowsum,
                           reinterpret_cast<float*>(W));   // W is free until the next pass
        else write_layout(Pm, slot, r, S, Spad, R, matw, matw_stride, layout, rowsum);
        __syncthreads();
    }
}

// Q = V diag(lambda) Vinv for a host-supplied eigensystem. One block.
__global__ void k_q_from_eigen(int S, int Spad, const double* __restrict__ V,
                               const double* __restrict__ Vinv, const double* __restrict__ lam,
                               double* __restrict__ Q) {
    for (int idx = threadIdx.x; idx < Spad * Spad; idx += blockDim.x) {
        int i = idx / Spad, j = idx % Spad;
        double acc = 0.0;
        if (i < S && j < S)
            for (int k = 0; k < S; ++k) acc += V[i * Spad + k] * lam[k] * Vinv[k * Spad + j];
        Q[idx] = acc;
    }
}

static int model_check_err(Instance* I, const char* what) {
    int h_err = 0;
    cudaError_t e = cudaMemcpyAsync(&h_err, I->d_err, sizeof(int), cudaMemcpyDeviceToHost, I->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(I->stream);
    if (e != cudaSuccess) return cuda_check(I, e, what);
    if (h_err) {
        cudaMemsetAsync(I->d_err, 0, sizeof(int), I->stream);
        return fail(I, TL_ERR_NUMERIC, "%s: device check %d failed (non-positive frequency, "
                    "zero mean rate or Jacobi did not converge)", what, h_err);
    }
    return TL_OK;
}

int launch_build_model(Instance* I, int m, int kind, const double* d_params, int n_params,
                       const double* d_freqs, int n_freqs, bool check) {
    (void)n_params;
    (void)n_freqs;
    ModelDev& M = I->models[m];
    int n_dq = kind == TL_MODEL_HKY ? 1 : kind == TL_MODEL_GTR ? 6
               : (kind == TL_MODEL_GY94 || kind == TL_MODEL_GY94RE) ? 2 : 0;
    M.n_dq = n_dq;
    k_build_model<<<1, 256, 0, I->stream>>>(kind, I->S, I->Spad, d_params, d_freqs, M.Q, M.pi,
                                            M.dQ, n_dq, M.pairs, M.mu, I->d_err);
    I->launches += 1;
    int rc = cuda_check(I, cudaGetLastError(), "build model");
    if (rc) return rc;
    if (check && (rc = model_check_err(I, "tl_set_model"))) return rc;
    return launch_eigen_from_q(I, m, check);
}

// above this many states the eigensystem's FP64 products run on many SMs
constexpr int kEigSplitS = 32;

int launch_eigen_from_q(Instance* I, int m, bool check) {
    ModelDev& M = I->models[m];
    M.basis_ready = false;   // V changes (and the basis area may serve as scratch)
    const size_t smem = 4 * 64 * 65 * sizeof(double) + 2 * 64 * 65 * sizeof(float);
    cudaFuncSetAttribute(k_eigen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (I->S <= kEigSplitS) {
        k_eigen<<<1, 256, smem, I->stream>>>(I->S, I->Spad, M.Q, M.pi, M.V, M.Vinv, M.lam,
                                             I->d_err, 0, nullptr);
        I->launches += 1;
    } else {
        // the parameter basis area is scratch here (the model change voids it)
        const int n = I->S, L = I->Spad;
        const size_t SS = (size_t)L * L;
        double* sA = M.G;
        double* sU = M.G + SS;
        double* s1 = M.G + 2 * SS;
        double* s2 = M.G + 3 * SS;
        k_eigen<<<1, kEigThreadsMax, smem, I->stream>>>(I->S, I->Spad, M.Q, M.pi, M.V, M.Vinv,
                                                        M.lam, I->d_err, 1, M.G);
        // two Newton-Schulz steps U <- U (3 I - U^T U) / 2, then U^T A U
        k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sU, sU, s1, 1, 1);
        k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sU, s1, s2, 0, 0);
        k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, s2, s2, s1, 1, 1);
        k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, s2, s1, sU, 0, 0);
        k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sA, sU, s1, 0, 0);
        k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sU, s1, s2, 1, 0);
        // two refinement steps, each: G = I + Theta (k_eig_rot), made
        // orthogonal by two Newton-Schulz steps, U <- U G, A <- G^T A G
        // (the second step writes back to U's and A's slots)
        double* sG = M.G + 4 * SS;
        double* sG2 = M.G + 5 * SS;
        double* alt[2][2] = {{M.G + 6 * SS, M.G + 7 * SS}, {sU, s2}};
        double *cu = sU, *ca = s2;
        for (int step = 0; step < 2; ++step) {
            double *nu = alt[step][0], *na = alt[step][1];
            k_eig_rot<<<n, 64, 0, I->stream>>>(n, L, ca, sG);
            k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sG, sG, s1, 1, 1);
            k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sG, s1, sG2, 0, 0);
            k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sG2, sG2, s1, 1, 1);
            k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sG2, s1, sG, 0, 0);
            k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, cu, sG, nu, 0, 0);
            k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, ca, sG, s1, 0, 0);
            k_eig_gemm<<<n, 64, 0, I->stream>>>(n, L, sG, s1, na, 1, 0);
            cu = nu;
            ca = na;
        }
        k_eigen<<<1, kEigThreadsMax, smem, I->stream>>>(I->S, I->Spad, M.Q, M.pi, M.V, M.Vinv,
                                                        M.lam, I->d_err, 2, M.G);
        I->launches += 8 + 2 * 8;
    }
    int rc = cuda_check(I, cudaGetLastError(), "eigen");
    if (rc) return rc;
    if (check && (rc = model_check_err(I, "eigendecomposition"))) return rc;
    return launch_model_working_copies(I, m);
}

int launch_param_basis(Instance* I, int m);

int launch_q_from_eigen(Instance* I, int m) {
    ModelDev& M = I->models[m];
    k_q_from_eigen<<<1, 256, 0, I->stream>>>(I->S, I->Spad, M.V, M.Vinv, M.lam, M.Q);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "Q from eigensystem");
}

int launch_model_working_copies(Instance* I, int m) {
    ModelDev& M = I->models[m];
    if (I->prec == kF64) {
        k_model_working<double><<<1, 256, 0, I->stream>>>(I->S, I->Spad, M.Q, M.pi,
                                                          (double*)M.Qw, (double*)M.piw, 0);
    } else {
        k_model_working<float><<<1, 256, 0, I->stream>>>(I->S, I->Spad, M.Q, M.pi,
                                                         (float*)M.Qw, (float*)M.piw,
                                                         I->prec == kTF32);
        // only the TF32 matrix layouts take the double-float products (the
        // four-state FP32 layout is formed from the FP64 eigensystem)
        if (!(I->S == 4 && I->prec == kF32)) {
            k_df_pairs<<<16, 256, 0, I->stream>>>(I->Spad * I->Spad, M.V, M.Vinv, (df2*)M.Vdf,
                                                  (df2*)M.Vinvdf);
            I->launches += 1;
        }
    }
    I->launches += 1;
    int rc = cuda_check(I, cudaGetLastError(), "model working copies");
    if (rc) return rc;
    if (I->prec == kTF32 && (rc = launch_q_tc(I, m))) return rc;
    M.basis_ready = false;  // computed by the first parameter-derivative request
    M.ready = true;
    return TL_OK;
}

int launch_update_matrices(Instance* I, int m, const int* d_pidx, const int* d_dpidx,
                           const double* d_len, int count) {
    if (count <= 0) return TL_OK;
    ModelDev& M = I->models[m];
    const double* d_rates = I->d_tmp;  // rates staged by the caller at d_tmp[0..R)
    dim3 grid(count, I->R);
    size_t smem = (128 + 3 * (size_t)I->Spad * I->Spad) * sizeof(double);
    int layout = (I->S == 4 && (I->prec == kF32 || I->prec == kF64)) ? 0
                 : (I->prec == kF64 ? 1 : (I->split ? 3 : 2));
    if (I->prec == kF64) {
        cudaFuncSetAttribute(k_tpm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tpm<double><<<grid, 256, smem, I->stream>>>(I->S, I->Spad, I->R, M.V, M.Vinv, nullptr,
                                                      nullptr, M.lam,
                                                      d_pidx, d_dpidx, d_len, d_rates, I->d_mat64,
                                                      (double*)I->d_matw, I->matw_stride, layout,
                                                      nullptr);
    } else {
        cudaFuncSetAttribute(k_tpm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_tpm<float><<<grid, 256, smem, I->stream>>>(I->S, I->Spad, I->R, M.V, M.Vinv,
                                                     (const df2*)M.Vdf, (const df2*)M.Vinvdf, M.lam,
                                                     d_pidx, d_dpidx, d_len, d_rates, I->d_mat64,
                                                     (float*)I->d_matw, I->matw_stride, layout,
                                                     I->d_rowsum);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "update matrices");
}


// G_k = Vinv dQ_k V for every parameter derivative of a model. One block per k.
// Two products of S^3 each, rows split over blockIdx.y: phase 0 writes
// W_k = dQ_k V into G, phase 1 overwrites G row by row with Vinv W_k (each
// block keeps W_k in shared memory, so rows of G can be written in place).
constexpr int kBasisRowBlocks = 8;
__global__ void k_param_basis(int S, int Spad, int phase, const double* __restrict__ V,
                              const double* __restrict__ Vinv, const double* __restrict__ dQ,
                              double* __restrict__ G, double* __restrict__ Wtmp) {
    extern __shared__ double sm_basis[];
    const int k = blockIdx.x;
    const int rows = (S + kBasisRowBlocks - 1) / kBasisRowBlocks;
    const int r0 = blockIdx.y * rows, r1 = min(S, r0 + rows);
    const size_t SS = (size_t)Spad * Spad;
    const double* L = phase == 0 ? dQ + k * SS : Vinv;   // left factor
    const double* Rt = phase == 0 ? V : Wtmp + k * SS;   // right factor
    double* out = phase == 0 ? Wtmp + k * SS : G + k * SS;
    double* Rs = sm_basis;  // the right factor, [S][Spad]
    for (int idx = threadIdx.x; idx < S * Spad; idx += blockDim.x) Rs[idx] = Rt[idx];
    __syncthreads();
    for (int idx = threadIdx.x; idx < (r1 - r0) * Spad; idx += blockDim.x) {
        const int i = r0 + idx / Spad, j = idx % Spad;
        double acc = 0.0;
        if (j < S)
            for (int a = 0; a < S; ++a) acc += L[i * Spad + a] * Rs[a * Spad + j];
        out[i * Spad + j] = acc;
    }
    if (blockIdx.y == 0)
        for (int idx = S * Spad + threadIdx.x; idx < Spad * Spad; idx += blockDim.x) out[idx] = 0.0;
}

// dP_r(t)/dtheta = V [G o Phi] Vinv with Phi_ij = rho t (e^{a_i} - e^{a_j}) / (a_i - a_j),
// a = rho t lambda (the Frechet derivative of the matrix exponential in the
// eigenbasis, Daleckii-Krein); grid (count, R).
template <typename T>
__global__ void k_param_tpm(int S, int Spad, int R, const double* __restrict__ V,
                            const double* __restrict__ Vinv, const double* __restrict__ lam,
                            const double* __restrict__ G, const int* __restrict__ idx_out,
                            const double* __restrict__ len, const double* __restrict__ rates,
                            double* __restrict__ mat64, T* __restrict__ matw, size_t matw_stride,
                            int layout, T* __restrict__ rowsum) {
    extern __shared__ double sm_ptpm[];
    double* X = sm_ptpm;                         // [Spad*Spad]
    double* Pm = sm_ptpm + (size_t)Spad * Spad;  // [Spad*Spad]
    __shared__ double a[64], ea[64];
    const int b = blockIdx.x, r = blockIdx.y;
    const int t = threadIdx.x, nt = blockDim.x;
    const double rt = rates[r] * len[b];
    const int slot = idx_out[b];
    for (int k = t; k < Spad; k += nt) {
        a[k] = (k < S) ? lam[k] * rt : 0.0;
        ea[k] = (k < S) ? exp(a[k]) : 0.0;
    }
    __syncthreads();
    for (int idx = t; idx < Spad * Spad; idx += nt) {
        const int i = idx / Spad, j = idx % Spad;
        double phi = 0.0;
        if (i < S && j < S) {
            const double d = a[i] - a[j];
            // (e^{a_i} - e^{a_j}) / (a_i - a_j) = e^{a_j} expm1(d) / d, -> e^{a_i} as d -> 0
            phi = (fabs(d) < 1e-12) ? ea[i] : ea[j] * expm1(d) / d;
        }
        X[idx] = rt * G[idx] * phi;
    }
    __syncthreads();
    // Pm = (V X) Vinv: Y = V X first (in Pm's place), then Y Vinv
    double* Y = X + 2 * (size_t)Spad * Spad;     // [Spad*Spad]
    for (int idx = t; idx < Spad * Spad; idx += nt) {
        const int i = idx / Spad, k = idx % Spad;
        double vx = 0.0;
        if (i < S && k < S)
            for (int l = 0; l < S; ++l) vx += V[i * Spad + l] * X[l * Spad + k];
        Y[idx] = vx;
    }
    __syncthreads();
    for (int idx = t; idx < Spad * Spad; idx += nt) {
        const int i = idx / Spad, j = idx % Spad;
        double acc = 0.0;
        if (i < S && j < S)
            for (int k = 0; k < S; ++k) acc += Y[i * Spad + k] * Vinv[k * Spad + j];
        Pm[idx] = acc;
        mat64[((size_t)slot * R + r) * Spad * Spad + idx] = acc;
    }
    __syncthreads();
    write_layout(Pm, slot, r, S, Spad, R, matw, matw_stride, layout, rowsum);
}

// G_k = Vinv dQ_k V, computed on first use after a model change (only the
// substitution-parameter derivatives need it). W_k = dQ_k V goes to the
// second half of the basis allocation ([2][kMaxDq][Spad][Spad]).
int launch_param_basis(Instance* I, int m) {
    ModelDev& M = I->models[m];
    if (M.n_dq == 0 || M.basis_ready) return TL_OK;
    const size_t SS = (size_t)I->Spad * I->Spad;
    const size_t smem = (size_t)I->S * I->Spad * sizeof(double);
    cudaFuncSetAttribute(k_param_basis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(M.n_dq, kBasisRowBlocks);
    double* W = M.G + SS * kMaxDq;
    for (int phase = 0; phase < 2; ++phase)
        k_param_basis<<<grid, 256, smem, I->stream>>>(I->S, I->Spad, phase, M.V, M.Vinv, M.dQ,
                                                      M.G, W);
    I->launches += 2;
    int rc = cuda_check(I, cudaGetLastError(), "parameter basis");
    if (!rc) M.basis_ready = true;
    return rc;
}

int launch_param_matrices(Instance* I, int m, int param, const int* d_idx, const double* d_len,
                          int count) {
    if (count <= 0) return TL_OK;
    ModelDev& M = I->models[m];
    int rc = launch_param_basis(I, m);
    if (rc) return rc;
    const double* d_rates = I->d_tmp;
    dim3 grid(count, I->R);
    const size_t smem = 3 * (size_t)I->Spad * I->Spad * sizeof(double);
    const int layout = (I->S == 4 && (I->prec == kF32 || I->prec == kF64)) ? 0
                       : (I->prec == kF64 ? 1 : (I->split ? 3 : 2));
    const double* G = M.G + (size_t)param * I->Spad * I->Spad;
    if (I->prec == kF64) {
        cudaFuncSetAttribute(k_param_tpm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_param_tpm<double><<<grid, 256, smem, I->stream>>>(
            I->S, I->Spad, I->R, M.V, M.Vinv, M.lam, G, d_idx, d_len, d_rates, I->d_mat64,
            (double*)I->d_matw, I->matw_stride, layout, nullptr);
    } else {
        cudaFuncSetAttribute(k_param_tpm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_param_tpm<float><<<grid, 256, smem, I->stream>>>(
            I->S, I->Spad, I->R, M.V, M.Vinv, M.lam, G, d_idx, d_len, d_rates, I->d_mat64,
            (float*)I->d_matw, I->matw_stride, layout, I->d_rowsum);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "parameter derivative matrices");
}

}  // namespace tl
