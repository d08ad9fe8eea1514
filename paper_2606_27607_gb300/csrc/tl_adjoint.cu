// Reverse-mode adjoint of the log-likelihood with respect to the transition
// matrices, the rate matrix and the substitution parameters.
//
// For an edge c (parent n, sibling s) and category r the pattern likelihood
// is linear in P_c,r: L_p = sum_r w_r u_c[r,p]^T P_c,r p_c[r,p] with
// u_c = q_n o (P_s p_s), q_n the parent's pre-order partial (Sec.
// "Algorithmic advances": pre-order partials; the likelihood is their inner
// product with the post-order partials at any node). Hence
//   M_c,r = dlogL/dP_c,r = w_r sum_p (w_p / L_p) u_c[r,p] p_c[r,p]^T .
// The accumulation kernels sum these outer products over patterns, one pass
// over q_n, p_a, p_b per parent; the finish works in the eigenbasis of Q:
// with W = V^T M V^-T and a = rho_r t_c lambda,
//   dlogL/dt_c = sum_r sum_i W_ii rho_r lambda_i e^{a_i},
//   G = sum_{c,r} rho_r t_c W o Phi,  Phi_ij = (e^{a_i} - e^{a_j}) / (a_i - a_j),
//   dlogL/dQ = V^-T G V^T,
// the adjoint of the Frechet derivative of the matrix exponential
// (Daleckii-Krein), so that every substitution parameter costs one S x S
// inner product <dlogL/dQ, dQ/dtheta> (Sec. "Discussion": exact
// substitution gradients in O(S^3 + N S^2) through the adjoint of the matrix
// exponential; Sec. "Algorithmic advances": the gradient for random-effects
// models as dlogL/dQ times dQ/dtheta, with a first-order approximation of
// the exponential's derivative, dP ~ rho t dQ P, kept here for comparison).
//
// The scales of u and p cancel against L_p's. The four-state kernel forms
// L_p from the same products, sum_r w_r q_n . (v_a o v_b) (all categories
// of a pattern in neighbouring lanes); for any S a first kernel takes it
// from the parent's stored post-order partial, L_p ~ 2^{s_n} sum_r w_r
// q_n . p_n, with s_n the parent's own rescaling exponent (its cumulative
// exponent minus its children's): one read of q_n and p_n instead of the
// two products per category. The stored p_n is v_a o v_b rounded to the
// working precision, so the two forms differ by that rounding (about 1e-5
// relative over 64 states for TF32 storage, 1e-16 in FP64).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "tl_df.cuh"
#include "tl_internal.cuh"

namespace tl {


__device__ __forceinline__ void load4(const float* p, float* o) {
    float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double* o) {
    double2 v = reinterpret_cast<const double2*>(p)[0];
    double2 w = reinterpret_cast<const double2*>(p)[1];
    o[0] = v.x; o[1] = v.y; o[2] = w.x; o[3] = w.y;
}

// ---- four states ------------------------------------------------------------
// Block: one parent, one chunk of patterns, four warps. A warp holds 32/LPP
// patterns with the R categories of a pattern in LPP neighbouring lanes, so
// L_p is a butterfly sum over those lanes. Each lane accumulates both
// children's 4 x 4 outer products for its category; the sums over a warp's
// patterns and then over the four warps are in a fixed order. Each lane
// streams its own q and child partials (16 or 32 bytes per pattern) through a
// kAdjStages-deep cp.async ring in shared memory, so that several patterns'
// loads are in flight per lane without holding registers.
constexpr int kAdjStages = 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename T, int LPP>
__global__ void __launch_bounds__(128) k_adj4(const AdjOp<T>* __restrict__ ops, AdjArgs a,
                                              double* __restrict__ mpart) {
    __shared__ T sP[2][kMaxCat][17];   // pitch 17: lanes of 4 categories hit 4 banks
    __shared__ T spi[4];
    __shared__ double red[4][kMaxCat][32];
    // ring: [warp][stage][array (q, x_a, x_b)][lane][4] (two stages in FP64: static
    // shared memory stays under 48 KB)
    constexpr int NST = sizeof(T) == 8 ? 2 : kAdjStages;
    __shared__ __align__(16) T ring[4][NST][3][32][4];
    const AdjOp<T>& op = ops[blockIdx.x];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int idx = t; idx < 2 * a.R * 16; idx += blockDim.x) {
        const int c = idx / (a.R * 16), rem = idx % (a.R * 16);
        sP[c][rem >> 4][rem & 15] = (T)op.P[c][rem];
    }
    if (t < 4) spi[t] = (T)a.pi[t];
    __syncthreads();
    constexpr int PPW = 32 / LPP;
    const int r = lane % LPP, ps = lane / LPP;
    const bool act = r < a.R;
    const int rr = act ? r : 0;
    const T wr = act ? (T)a.catw[r] : T(0);
    const int p_begin = blockIdx.y * a.chunk;
    const int p_end = min(a.Ppad, p_begin + a.chunk);
    // the op's pointers in registers (the copies' memory clobbers would
    // otherwise reload them every pattern)
    const T* q = op.q;
    const int8_t* st[2] = {op.st[0], op.st[1]};
    const T* part[2] = {op.part[0], op.part[1]};
    const double* patw = a.patw;
    const bool st0 = st[0] != nullptr, st1 = st[1] != nullptr;
    T accA[16], accB[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) accA[k] = accB[k] = T(0);
    bool bad = false;
    const int first = p_begin + warp * PPW, step = 4 * PPW;
    const int n_it = first < p_end ? (p_end - first + step - 1) / step : 0;
    // issue the copies of iteration k into its stage (an empty group past the end)
    auto issue = [&](int k) {
        if (k < n_it) {
            const int p = first + k * step + ps;
            const int pl = p < p_end ? p : p_begin;
            const size_t off = ((size_t)rr * a.Ppad + pl) * 4;
            T(*stg)[32][4] = ring[warp][k % NST];
#pragma unroll
            for (int h = 0; h < (int)sizeof(T) * 4 / 16; ++h) {
                if (q) cp_async16(&stg[0][lane][h * 16 / sizeof(T)], q + off + h * 16 / sizeof(T));
                if (!st0) cp_async16(&stg[1][lane][h * 16 / sizeof(T)],
                                     part[0] + off + h * 16 / sizeof(T));
                if (!st1) cp_async16(&stg[2][lane][h * 16 / sizeof(T)],
                                     part[1] + off + h * 16 / sizeof(T));
            }
        }
        cp_async_commit();
    };
    // tip states and pattern weights: registers, one pattern ahead
    int nst[2] = {0, 0};
    double nwp = 0.0;
    auto fetch_small = [&](int k) {
        const int p = first + k * step + ps;
        const int pl = p < p_end ? p : p_begin;
        if (st0) nst[0] = st[0][pl];
        if (st1) nst[1] = st[1][pl];
        nwp = p < p_end ? patw[pl] : 0.0;
    };
#pragma unroll
    for (int k = 0; k < NST - 1; ++k) issue(k);
    if (n_it > 0) fetch_small(0);
    for (int k = 0; k < n_it; ++k) {
        issue(k + NST - 1);
        const int sv[2] = {nst[0], nst[1]};
        const double wp = nwp;
        if (k + 1 < n_it) fetch_small(k + 1);
        cp_async_wait<NST - 1>();
        const int p = first + k * step + ps;
        const bool inb = p < p_end;
        const T(*stg)[32][4] = ring[warp][k % NST];
        T qv[4], x[2][4], v[2][4];
        if (q) load4(&stg[0][lane][0], qv);
        else {
#pragma unroll
            for (int i = 0; i < 4; ++i) qv[i] = spi[i];
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (c == 0 ? st0 : st1) {
                const int s = sv[c];
                const bool amb = s < 0 || s >= 4;
#pragma unroll
                for (int j = 0; j < 4; ++j) x[c][j] = (amb || s == j) ? T(1) : T(0);
            } else {
                load4(&stg[1 + c][lane][0], x[c]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                T s = T(0);
#pragma unroll
                for (int j = 0; j < 4; ++j) s += sP[c][rr][i * 4 + j] * x[c][j];
                v[c][i] = s;
            }
        }
        T d = T(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) d += qv[i] * v[0][i] * v[1][i];
        d = (act && inb) ? wr * d : T(0);
#pragma unroll
        for (int o = 1; o < LPP; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        T coef = T(0);
        if (wp != 0.0) {
            if (d > T(0)) coef = (T)wp / d;
            else bad = true;
        }
        const T cw = coef * wr;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const T ua = cw * qv[i] * v[1][i], ub = cw * qv[i] * v[0][i];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                accA[i * 4 + j] += ua * x[0][j];
                accB[i * 4 + j] += ub * x[1][j];
            }
        }
    }
    cp_async_wait<0>();
    if (bad) atomicOr(a.err, 1);
#pragma unroll
    for (int o = LPP; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            accA[k] += __shfl_xor_sync(0xffffffffu, accA[k], o);
            accB[k] += __shfl_xor_sync(0xffffffffu, accB[k], o);
        }
    }
    if (ps == 0 && act) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            red[warp][r][k] = (double)accA[k];
            red[warp][r][16 + k] = (double)accB[k];
        }
    }
    __syncthreads();
    for (int idx = t; idx < a.R * 32; idx += blockDim.x) {
        const int rc = idx >> 5, k = idx & 31, c = k >> 4;
        const double s = ((red[0][rc][k] + red[1][rc][k]) + red[2][rc][k]) + red[3][rc][k];
        const int row = op.row[c];
        if (row >= 0)
            mpart[(size_t)blockIdx.y * a.n_rows + (size_t)(row * a.R + rc) * 16 + (k & 15)] = s;
    }
}

// ---- any S <= 64: the outer products as two small GEMMs per tile ----------
// Block: one parent, one category, one chunk of patterns; 256 threads; tiles
// of 32 patterns x 64 states (states beyond S are zero). Per tile:
//   v_c = p_c P_c^T            (thread: 4 patterns x 4 states of one child)
//   U_a = coef w_r q o v_b, U_b = coef w_r q o v_a
//   M_a += U_a^T p_a, M_b += U_b^T p_b   (thread: a 4 x 4 block of each)
constexpr int kGT = 32;       // patterns per tile
constexpr int kGP = 36;       // row pitch of the transposed tiles (16-byte rows)
// Stage one tile of category r: q (pi at the root), both children's
// partials row-major (X) and transposed (XT); states beyond S are zero.
template <typename T>
__device__ __forceinline__ void adj_load_tile(const AdjOp<T>& op, const AdjArgs& a, int r, int p0,
                                              T* X, T* XT, T* Qs) {
    const int S = a.S, Spad = a.Spad;
    for (int idx = threadIdx.x; idx < kGT * 64; idx += blockDim.x) {
        const int pp = idx >> 6, j = idx & 63, p = p0 + pp;
        const size_t off = ((size_t)r * a.Ppad + p) * Spad + j;
        T qv = T(0);
        if (j < S) qv = op.q ? op.q[off] : (T)a.pi[j];
        Qs[idx] = qv;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            T xv = T(0);
            if (j < S) {
                if (op.st[c]) {
                    const int s = op.st[c][p];
                    xv = (s < 0 || s >= S || s == j) ? T(1) : T(0);
                } else {
                    xv = op.part[c][off];
                }
            }
            if (X) X[c * kGT * 64 + idx] = xv;
            XT[(c * 64 + j) * kGP + pp] = xv;
        }
    }
}

// Both children's P_c,r, transposed: Pt[c][j][i] = P_c,r[i][j].
template <typename T>
__device__ __forceinline__ void adj_load_mats(const AdjOp<T>& op, const AdjArgs& a, int r, T* Pt) {
    const int S = a.S, Spad = a.Spad;
    for (int idx = threadIdx.x; idx < 2 * 64 * 64; idx += blockDim.x) {
        const int c = idx >> 12, j = (idx >> 6) & 63, i = idx & 63;
        Pt[idx] = (i < S && j < S) ? (T)op.P[c][((size_t)r * Spad + i) * Spad + j] : T(0);
    }
}

// v_c = p_c P_c^T for both children (256 threads: thread = child, 4
// patterns, 4 states), into Vs[c][p][i].
template <typename T>
__device__ __forceinline__ void adj_tile_v(const T* Pt, const T* XT, T* Vs) {
    const int t = threadIdx.x;
    const int vc = t >> 7, vp = ((t & 127) >> 4) * 4, vi = (t & 15) * 4;
    T acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = T(0);
    const T* pw = Pt + vc * 64 * 64 + vi;
    const T* px = XT + vc * 64 * kGP + vp;
#pragma unroll 8
    for (int j = 0; j < 64; ++j) {
        T w4[4], x4[4];
        load4(pw + j * 64, w4);
        load4(px + j * kGP, x4);
#pragma unroll
        for (int pp = 0; pp < 4; ++pp)
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) acc[pp * 4 + ii] += x4[pp] * w4[ii];
    }
#pragma unroll
    for (int pp = 0; pp < 4; ++pp)
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) Vs[(vc * kGT + vp + pp) * 64 + vi + ii] = acc[pp * 4 + ii];
}

// w_p / L_p per parent and pattern from the stored q_n and p_n. Block: one
// parent, 16 patterns; a half-warp per pattern, a lane per four states
// (one 16-byte load of q and of p_n per category), fixed-order shuffle sums.
constexpr int kCoefPat = 16;
template <typename T>
__global__ void __launch_bounds__(256) k_adj_coef(const AdjOp<T>* __restrict__ ops, AdjArgs a,
                                                  double* __restrict__ coef) {
    const AdjOp<T>& op = ops[blockIdx.x];
    const int lane = threadIdx.x & 31, half = threadIdx.x >> 4, l16 = lane & 15;
    const int p = blockIdx.y * kCoefPat + half;
    const bool inb = p < a.Ppad;
    const int pl = inb ? p : 0;
    // FP32 instances sum the categories in FP32 (FP64 issue is a small fraction
    // of FP32 on this part; the coefficient feeds TF32 products), FP64 ones in FP64
    using Acc = typename std::conditional<sizeof(T) == 4, float, double>::type;
    Acc den = Acc(0);
    for (int r = 0; r < a.R; ++r) {
        T s = T(0);
        for (int i0 = 4 * l16; i0 < a.Spad; i0 += 64) {
            const size_t off = ((size_t)r * a.Ppad + pl) * a.Spad + i0;
            T q4[4], p4[4];
            if (op.q) load4(op.q + off, q4);
            else {
#pragma unroll
                for (int k = 0; k < 4; ++k) q4[k] = i0 + k < a.S ? (T)a.pi[i0 + k] : T(0);
            }
            load4(op.pn + off, p4);
#pragma unroll
            for (int k = 0; k < 4; ++k) s += q4[k] * p4[k];
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        den += (Acc)a.catw[r] * (Acc)s;
    }
    if (l16 == 0 && inb) {
        const double wp = a.patw[p];
        double cf = 0.0;
        if (wp != 0.0) {
            int sn = op.en ? op.en[p] : 0;
            for (int c = 0; c < 2; ++c) sn -= op.ec[c] ? op.ec[c][p] : 0;
            if (den > Acc(0)) cf = ldexp((double)((Acc)wp / den), -sn);
            else atomicOr(a.err, 1);
        }
        coef[(size_t)blockIdx.x * a.Ppad + p] = cf;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_adj_gen(const AdjOp<T>* __restrict__ ops, AdjArgs a,
                                                 double* __restrict__ mpart) {
    extern __shared__ __align__(16) unsigned char sm_adj[];
    T* Pt = reinterpret_cast<T*>(sm_adj);        // [2][64][64]: Pt[c][j][i] = P_c[i][j]
    T* X = Pt + 2 * 64 * 64;                     // [2][kGT][64] child partials
    T* XT = X + 2 * kGT * 64;                    // [2][64][kGP] transposed
    T* Qs = XT + 2 * 64 * kGP;                   // [kGT][64]
    T* Vs = Qs + kGT * 64;                       // [2][kGT][64] v, then U
    T* Cs = Vs + 2 * kGT * 64;                   // [kGT] coef w_r
    const AdjOp<T>& op = ops[blockIdx.x];
    const int r = blockIdx.y;
    const int t = threadIdx.x;
    const int Spad = a.Spad;
    adj_load_mats(op, a, r, Pt);
    const T wr = (T)a.catw[r];
    const int p_begin = blockIdx.z * a.chunk;
    const int p_end = min(a.Ppad, p_begin + a.chunk);
    const int mi = (t >> 4) * 4, mj = (t & 15) * 4;
    T accA[16], accB[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) accA[k] = accB[k] = T(0);
    for (int p0 = p_begin; p0 < p_end; p0 += kGT) {
        __syncthreads();  // the previous tile's readers are done
        adj_load_tile(op, a, r, p0, X, XT, Qs);
        if (t < kGT) Cs[t] = (T)a.coef[(size_t)blockIdx.x * a.Ppad + p0 + t] * wr;
        __syncthreads();
        adj_tile_v(Pt, XT, Vs);
        __syncthreads();
        for (int idx = t; idx < kGT * 64; idx += blockDim.x) {
            const T qc = Qs[idx] * Cs[idx >> 6];
            const T va = Vs[idx], vb = Vs[kGT * 64 + idx];
            Vs[idx] = qc * vb;               // U_a
            Vs[kGT * 64 + idx] = qc * va;    // U_b
        }
        __syncthreads();
#pragma unroll 4
        for (int pp = 0; pp < kGT; ++pp) {
            T ua[4], ub[4], xa[4], xb[4];
            load4(Vs + pp * 64 + mi, ua);
            load4(Vs + (kGT + pp) * 64 + mi, ub);
            load4(X + pp * 64 + mj, xa);
            load4(X + (kGT + pp) * 64 + mj, xb);
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    accA[ii * 4 + jj] += ua[ii] * xa[jj];
                    accB[ii * 4 + jj] += ub[ii] * xb[jj];
                }
        }
    }
    const int SS = Spad * Spad;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int row = op.row[c];
        if (row < 0) continue;
        const T* acc = c ? accB : accA;
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int i = mi + ii, j = mj + jj;
                if (i < Spad && j < Spad)
                    mpart[(size_t)blockIdx.z * a.n_rows + (size_t)(row * a.R + r) * SS + i * Spad + j] =
                        (double)acc[ii * 4 + jj];
            }
    }
}

static size_t adj_gen_smem(int elt) {
    return (size_t)elt * (2 * 64 * 64 + 2 * kGT * 64 + 2 * 64 * kGP + kGT * 64 + 2 * kGT * 64 + kGT);
}

static bool adj_nuc(const Instance* I) { return I->S == 4 && (I->prec == kF32 || I->prec == kF64); }
static bool adj_tc(const Instance* I) { return I->prec == kTF32 && I->Spad == 64; }
static int adj_lpp(int R) { return R <= 1 ? 1 : R <= 2 ? 2 : R <= 4 ? 4 : 8; }

// Pattern chunks per parent: enough blocks for a few waves on the device,
// and chunks short enough that an FP32 accumulator sums a bounded number of
// positive terms (at most 4,096 patterns per chunk).
int adj_chunks(const Instance* I, int n_ops) {
    const int sms = 152;
    const int per = adj_nuc(I) ? n_ops : n_ops * I->R;
    const int step = (adj_nuc(I) || adj_tc(I)) ? 128 : kGT;
    int n = std::max(1, (4 * sms + per - 1) / std::max(per, 1));
    const int cap = adj_nuc(I) ? (I->elt == 4 ? 2048 : (1 << 30)) : 4096;
    n = std::max(n, (I->Ppad + cap - 1) / cap);
    n = std::min(n, (I->Ppad + step - 1) / step);
    return n;
}

static int adj_chunk_len(const Instance* I, int n_chunks) {
    const int step = (adj_nuc(I) || adj_tc(I)) ? 128 : kGT;
    const int len = (I->Ppad + n_chunks - 1) / n_chunks;
    return ((len + step - 1) / step) * step;
}

template <typename T>
static int adj_accumulate_t(Instance* I, const void* d_ops, int n_ops, int n_chunks,
                            size_t n_rows, double* d_coef, double* d_mpart, int model) {
    AdjArgs a;
    a.pi = I->models[model].pi;
    a.patw = I->d_patw;
    a.coef = d_coef;
    a.err = I->d_err + 1;
    a.timeout = I->d_err + 2;
    a.R = I->R;
    a.Ppad = I->Ppad;
    a.Spad = I->Spad;
    a.S = I->S;
    a.n_chunks = n_chunks;
    a.n_rows = n_rows;
    a.chunk = adj_chunk_len(I, n_chunks);
    for (int r = 0; r < kMaxCat; ++r) a.catw[r] = r < I->R ? I->h_catw[r] : 0.0;
    const AdjOp<T>* ops = reinterpret_cast<const AdjOp<T>*>(d_ops);
    if (adj_nuc(I)) {
        dim3 grid(n_ops, n_chunks);
        switch (adj_lpp(I->R)) {
            case 1: k_adj4<T, 1><<<grid, 128, 0, I->stream>>>(ops, a, d_mpart); break;
            case 2: k_adj4<T, 2><<<grid, 128, 0, I->stream>>>(ops, a, d_mpart); break;
            case 4: k_adj4<T, 4><<<grid, 128, 0, I->stream>>>(ops, a, d_mpart); break;
            default: k_adj4<T, 8><<<grid, 128, 0, I->stream>>>(ops, a, d_mpart); break;
        }
        I->launches += 1;
        return cuda_check(I, cudaGetLastError(), "adjoint (four states)");
    }
    k_adj_coef<T><<<dim3(n_ops, (I->Ppad + kCoefPat - 1) / kCoefPat), 256, 0, I->stream>>>(
        ops, a, d_coef);
    if (adj_tc(I)) {
        I->launches += 1;
        if (int rc = cuda_check(I, cudaGetLastError(), "adjoint coefficients")) return rc;
        return launch_adj_tc(I, reinterpret_cast<const AdjOp<float>*>(d_ops), n_ops, n_chunks, a,
                             d_mpart);
    }
    const size_t smem = adj_gen_smem(sizeof(T));
    if constexpr (sizeof(T) == 8) {  // FP64 instances; FP32 storage is four-state or TF32
        cudaFuncSetAttribute(k_adj_gen<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_adj_gen<T><<<dim3(n_ops, I->R, n_chunks), 256, smem, I->stream>>>(ops, a, d_mpart);
    } else {
        return fail(I, TL_ERR_UNSUPPORTED, "adjoint: no kernel for this precision and S");
    }
    I->launches += 2;
    return cuda_check(I, cudaGetLastError(), "adjoint (any S)");
}

int launch_adj_accumulate(Instance* I, const void* d_ops, int n_ops, int n_chunks, size_t n_rows,
                          double* d_coef, double* d_mpart, int model) {
    if (I->Spad > 64) return fail(I, TL_ERR_UNSUPPORTED, "adjoint built for at most 64 states");
    if (I->elt == 8)
        return adj_accumulate_t<double>(I, d_ops, n_ops, n_chunks, n_rows, d_coef, d_mpart, model);
    return adj_accumulate_t<float>(I, d_ops, n_ops, n_chunks, n_rows, d_coef, d_mpart, model);
}

// out[row] = sum over chunks of in[chunk][row], in chunk order.
__global__ void k_sum_chunks(const double* __restrict__ in, size_t n_rows, int n_chunks,
                             double* __restrict__ out) {
    for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < n_rows;
         row += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < n_chunks; ++c) s += in[(size_t)c * n_rows + row];
        out[row] = s;
    }
}

int launch_adj_sum_chunks(Instance* I, const double* d_in, size_t n_rows, int n_chunks,
                          double* d_out) {
    if (n_rows == 0) return TL_OK;
    const int blocks = (int)std::min<size_t>((n_rows + 255) / 256, 152 * 16);
    k_sum_chunks<<<blocks, 256, 0, I->stream>>>(d_in, n_rows, n_chunks, d_out);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "adjoint chunk sums");
}

// ---- the finish in the eigenbasis, one block per edge ----------------------
// For each category: Y = V^T M, W = Y V^-T; the edge's branch derivative
// from diag(W); its share of G (exact: rho t W o Phi; first order:
// rho t M P^T in the original basis). FP64 for every precision: V of a
// codon model spans 1/sqrt(pi_min) (F3x4 frequencies reach 1e-4 and less),
// and the eigenbasis transform in FP32 amplified the rounding of M past the
// FP32 path's tolerance. Gpart is [Spad*Spad][E] for a fixed-order sum
// over edges.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_finish(int S, int Spad, int R, int E,
                                                    const double* __restrict__ V,
                                                    const double* __restrict__ Vinv,
                                                    const double* __restrict__ lam,
                                                    const double* __restrict__ rates,
                                                    const double* __restrict__ Mall,
                                                    const AdjEdge* __restrict__ edges,
                                                    int first_order, double* __restrict__ gpart,
                                                    double* __restrict__ grad) {
    // 256 threads as a 16 x 16 grid; thread (ti, tj) owns the 4 x 4 block of
    // rows 4 ti.. and columns 4 tj.. of Y and W (padded to 64 x 64, entries
    // beyond S are zero), so each shared-memory value it reads feeds four
    // multiply-adds
    extern __shared__ __align__(16) unsigned char sm_fin[];
    constexpr int L = 64, LP = 65;           // padded size, row pitch
    T* Vs = reinterpret_cast<T*>(sm_fin);    // [L][LP]
    T* Vi = Vs + L * LP;
    T* Ms = Vi + L * LP;
    T* Ys = Ms + L * LP;
    __shared__ double ea[64], la[64], gsum[8];
    const int e = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
    const int ti = t >> 4, tj = t & 15;
    const int SS = Spad * Spad;
    const AdjEdge ed = edges[e];
    for (int idx = t; idx < L * L; idx += nt) {
        const int i = idx >> 6, j = idx & 63;
        const bool in = i < S && j < S;
        Vs[i * LP + j] = in ? (T)V[i * Spad + j] : T(0);
        Vi[i * LP + j] = in ? (T)Vinv[i * Spad + j] : T(0);
    }
    double g[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) g[a][b] = 0.0;
    double dsum = 0.0;
    for (int r = 0; r < R; ++r) {
        const double rt = rates[r] * ed.t;
        __syncthreads();
        for (int idx = t; idx < L * L; idx += nt) {
            const int i = idx >> 6, j = idx & 63;
            Ms[i * LP + j] = (i < S && j < S) ? (T)Mall[((size_t)e * R + r) * SS + i * Spad + j]
                                             : T(0);
        }
        if (t < 64) {
            la[t] = t < S ? lam[t] * rt : 0.0;
            ea[t] = t < S ? exp(la[t]) : 0.0;
        }
        __syncthreads();
        // Y = V^T M: Y[i][l] = sum_k V[k][i] M[k][l]
        T y[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) y[a][b] = T(0);
        for (int k = 0; k < S; ++k) {
            T va[4], mb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) va[a] = Vs[k * LP + 4 * ti + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) mb[b] = Ms[k * LP + 4 * tj + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) y[a][b] += va[a] * mb[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Ys[(4 * ti + a) * LP + 4 * tj + b] = y[a][b];
        __syncthreads();
        // W = Y V^-T: W[i][j] = sum_l Y[i][l] Vinv[j][l]
        T wv[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) wv[a][b] = T(0);
        for (int l = 0; l < S; ++l) {
            T ya[4], vb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) ya[a] = Ys[(4 * ti + a) * LP + l];
#pragma unroll
            for (int b = 0; b < 4; ++b) vb[b] = Vi[(4 * tj + b) * LP + l];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) wv[a][b] += ya[a] * vb[b];
        }
        // the edge derivative (diagonal of W) and this edge's share of G
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = 4 * ti + a, j = 4 * tj + b;
                if (i >= S || j >= S) continue;
                const double w = (double)wv[a][b];
                if (i == j) dsum += w * rates[r] * lam[i] * ea[i];
                if (!first_order) {
                    const double d = la[i] - la[j];
                    const double phi = (fabs(d) < 1e-12) ? ea[i] : ea[j] * expm1(d) / d;
                    g[a][b] += rt * w * phi;
                } else {
                    const double* P = ed.P + (size_t)r * SS;
                    double mp = 0.0;
                    for (int l = 0; l < S; ++l) mp += (double)Ms[i * LP + l] * P[j * Spad + l];
                    g[a][b] += rt * mp;
                }
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = 4 * ti + a, j = 4 * tj + b;
            if (i < Spad && j < Spad) gpart[(size_t)(i * Spad + j) * E + e] = g[a][b];
        }
    // fixed-order block sum of the diagonal terms
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((t & 31) == 0) gsum[t >> 5] = dsum;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) s += gsum[w];
        grad[e] = s;
    }
}

// The finish of a TF32 instance with the two eigenbasis products in
// double-float arithmetic (tl_df.cuh): every value of V, V^-1, M and Y as
// hi + lo. W then enters the same FP64 arithmetic as the FP64 kernel, with
// Phi_ij = (e^{a_i} - e^{a_j}) / (a_i - a_j) from the exponentials (a series
// in d = a_i - a_j below |d| = 2^-10).
__global__ void __launch_bounds__(256) k_adj_finish_df(int S, int Spad, int R, int E,
                                                       const double* __restrict__ V,
                                                       const double* __restrict__ Vinv,
                                                       const double* __restrict__ lam,
                                                       const double* __restrict__ rates,
                                                       const double* __restrict__ Mall,
                                                       const AdjEdge* __restrict__ edges,
                                                       int first_order, double* __restrict__ gpart,
                                                       double* __restrict__ grad) {
    extern __shared__ __align__(16) unsigned char sm_fin[];
    constexpr int L = 64, LP = 65;
    df2* Vs = reinterpret_cast<df2*>(sm_fin);   // [L][LP]
    df2* Vi = Vs + L * LP;
    df2* Ms = Vi + L * LP;
    df2* Ys = Ms + L * LP;
    __shared__ double ea[64], la[64], gsum[8];
    const int e = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
    const int ti = t >> 4, tj = t & 15;
    const int SS = Spad * Spad;
    const AdjEdge ed = edges[e];
    for (int idx = t; idx < L * L; idx += nt) {
        const int i = idx >> 6, j = idx & 63;
        const bool in = i < S && j < S;
        Vs[i * LP + j] = df_of(in ? V[i * Spad + j] : 0.0);
        Vi[i * LP + j] = df_of(in ? Vinv[i * Spad + j] : 0.0);
    }
    double g[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) g[a][b] = 0.0;
    double dsum = 0.0;
    for (int r = 0; r < R; ++r) {
        const double rt = rates[r] * ed.t;
        __syncthreads();
        for (int idx = t; idx < L * L; idx += nt) {
            const int i = idx >> 6, j = idx & 63;
            Ms[i * LP + j] =
                df_of((i < S && j < S) ? Mall[((size_t)e * R + r) * SS + i * Spad + j] : 0.0);
        }
        if (t < 64) {
            la[t] = t < S ? lam[t] * rt : 0.0;
            ea[t] = t < S ? exp(la[t]) : 0.0;
        }
        __syncthreads();
        // Y = V^T M: Y[i][l] = sum_k V[k][i] M[k][l]
        float ys[4][4], yc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) ys[a][b] = yc[a][b] = 0.f;
        for (int k = 0; k < S; ++k) {
            df2 va[4], mb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) va[a] = Vs[k * LP + 4 * ti + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) mb[b] = Ms[k * LP + 4 * tj + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) df_mac(ys[a][b], yc[a][b], va[a], mb[b]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) Ys[(4 * ti + a) * LP + 4 * tj + b] = df_norm(ys[a][b], yc[a][b]);
        __syncthreads();
        // W = Y V^-T: W[i][j] = sum_l Y[i][l] Vinv[j][l]
        float ws[4][4], wc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) ws[a][b] = wc[a][b] = 0.f;
        for (int l = 0; l < S; ++l) {
            df2 ya[4], vb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) ya[a] = Ys[(4 * ti + a) * LP + l];
#pragma unroll
            for (int b = 0; b < 4; ++b) vb[b] = Vi[(4 * tj + b) * LP + l];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) df_mac(ws[a][b], wc[a][b], ya[a], vb[b]);
        }
        // the edge derivative (diagonal of W) and this edge's share of G
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = 4 * ti + a, j = 4 * tj + b;
                if (i >= S || j >= S) continue;
                const double w = (double)ws[a][b] + (double)wc[a][b];
                if (i == j) dsum += w * rates[r] * lam[i] * ea[i];
                if (!first_order) {
                    const double d = la[i] - la[j];
                    const double phi =
                        fabs(d) < 0x1p-10
                            ? ea[j] * (1.0 + d * (0.5 + d * (1.0 / 6 + d * (1.0 / 24 + d * (1.0 / 120)))))
                            : (ea[i] - ea[j]) / d;
                    g[a][b] += rt * w * phi;
                } else {
                    const double* P = ed.P + (size_t)r * SS;
                    double mp = 0.0;
                    for (int l = 0; l < S; ++l) {
                        const df2 m = Ms[i * LP + l];
                        mp += ((double)m.hi + (double)m.lo) * P[j * Spad + l];
                    }
                    g[a][b] += rt * mp;
                }
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = 4 * ti + a, j = 4 * tj + b;
            if (i < Spad && j < Spad) gpart[(size_t)(i * Spad + j) * E + e] = g[a][b];
        }
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((t & 31) == 0) gsum[t >> 5] = dsum;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) s += gsum[w];
        grad[e] = s;
    }
}

// Small state spaces (S <= 16): a thread per entry of Y and W.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_finish_small(int S, int Spad, int R, int E,
                                                    const double* __restrict__ V,
                                                    const double* __restrict__ Vinv,
                                                    const double* __restrict__ lam,
                                                    const double* __restrict__ rates,
                                                    const double* __restrict__ Mall,
                                                    const AdjEdge* __restrict__ edges,
                                                    int first_order, double* __restrict__ gpart,
                                                    double* __restrict__ grad) {
    extern __shared__ __align__(16) unsigned char sm_fin[];
    const int SS = Spad * Spad;
    T* Vs = reinterpret_cast<T*>(sm_fin);   // [Spad][Spad]
    T* Vi = Vs + SS;
    T* Ms = Vi + SS;
    T* Ys = Ms + SS;
    __shared__ double ea[64], la[64], gsum[8];
    const int e = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
    const AdjEdge ed = edges[e];
    for (int idx = t; idx < SS; idx += nt) {
        Vs[idx] = (T)V[idx];
        Vi[idx] = (T)Vinv[idx];
    }
    double g_acc[16];   // this thread's share of G (idx = t + k nt)
#pragma unroll
    for (int k = 0; k < 16; ++k) g_acc[k] = 0.0;
    double dsum = 0.0;
    for (int r = 0; r < R; ++r) {
        const double rt = rates[r] * ed.t;
        __syncthreads();
        for (int idx = t; idx < SS; idx += nt) Ms[idx] = (T)Mall[((size_t)e * R + r) * SS + idx];
        if (t < Spad) {
            la[t] = t < S ? lam[t] * rt : 0.0;
            ea[t] = t < S ? exp(la[t]) : 0.0;
        }
        __syncthreads();
        // Y = V^T M
        for (int idx = t; idx < SS; idx += nt) {
            const int i = idx / Spad, l = idx % Spad;
            T acc = T(0);
            for (int k = 0; k < S; ++k) acc += Vs[k * Spad + i] * Ms[k * Spad + l];
            Ys[idx] = acc;
        }
        __syncthreads();
        // W = Y V^-T, the edge derivative and G
        for (int k = 0, idx = t; idx < SS; ++k, idx += nt) {
            const int i = idx / Spad, j = idx % Spad;
            if (i >= S || j >= S) continue;
            T w = T(0);
            for (int l = 0; l < S; ++l) w += Ys[i * Spad + l] * Vi[j * Spad + l];
            if (i == j) dsum += (double)w * rates[r] * lam[i] * ea[i];
            if (!first_order) {
                const double d = la[i] - la[j];
                const double phi = (fabs(d) < 1e-12) ? ea[i] : ea[j] * expm1(d) / d;
                g_acc[k] += rt * (double)w * phi;
            } else {
                const double* P = ed.P + (size_t)r * SS;
                double mp = 0.0;
                for (int l = 0; l < S; ++l) mp += (double)Ms[i * Spad + l] * P[j * Spad + l];
                g_acc[k] += rt * mp;
            }
        }
    }
    for (int k = 0, idx = t; idx < SS; ++k, idx += nt) gpart[(size_t)idx * E + e] = g_acc[k];
    // fixed-order block sum of the diagonal terms
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
    if ((t & 31) == 0) gsum[t >> 5] = dsum;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < (nt >> 5); ++w) s += gsum[w];
        grad[e] = s;
    }
}

int launch_adj_finish(Instance* I, int model, const double* d_M, const AdjEdge* d_edges, int E,
                      bool first_order, double* d_gpart, double* d_grad) {
    if (E <= 0) return TL_OK;
    ModelDev& M = I->models[model];
    const int SS = I->Spad * I->Spad;
    if (SS > 16 * 256) return fail(I, TL_ERR_UNSUPPORTED, "adjoint built for at most 64 states");
    const double* d_rates = I->d_tmp;  // staged by the caller
    if (I->Spad <= 16) {
        const size_t smem = 4 * (size_t)SS * sizeof(double);
        k_adj_finish_small<double><<<E, 256, smem, I->stream>>>(
            I->S, I->Spad, I->R, E, M.V, M.Vinv, M.lam, d_rates, d_M, d_edges, first_order,
            d_gpart, d_grad);
    } else if (I->prec == kTF32 && !first_order) {
        const size_t smem = 4 * (size_t)64 * 65 * sizeof(df2);
        cudaFuncSetAttribute(k_adj_finish_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_adj_finish_df<<<E, 256, smem, I->stream>>>(I->S, I->Spad, I->R, E, M.V, M.Vinv, M.lam,
                                                     d_rates, d_M, d_edges, first_order, d_gpart,
                                                     d_grad);
    } else {
        const size_t smem = 4 * (size_t)64 * 65 * sizeof(double);
        cudaFuncSetAttribute(k_adj_finish<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        k_adj_finish<double><<<E, 256, smem, I->stream>>>(I->S, I->Spad, I->R, E, M.V, M.Vinv,
                                                          M.lam, d_rates, d_M, d_edges,
                                                          first_order, d_gpart, d_grad);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "adjoint finish");
}

// ---- dlogL/dQ and the parameters (one block, FP64) ---------------------------
// dQ = V^-T G V^T (G from the exact finish; the first-order finish already
// sums in the original basis), then <dQ, dQ/dtheta_k> for the model's
// stored derivatives and, for random effects on pair (i, j) of the
// normalised reversible Q,
//   dlogL/deps = Q_ij (dQ_ij - dQ_ii) + Q_ji (dQ_ji - dQ_jj)
//                - (pi_i Q_ij + pi_j Q_ji) <dQ, Q>
// (the derivative of exp(eps) s_ij pi_j and of the normaliser).
// dlogL/dQ = V^-T G V^T (exact form) or G itself (first order): block i forms
// row i, Y_i = sum_k Vinv[k][i] G[k][.], then D[i][j] = sum_l Y_i[l] V[j][l]
// (a thread per column; the rows run on separate SMs).
__global__ void __launch_bounds__(64) k_adj_dq(int S, int Spad, const double* __restrict__ V,
                                               const double* __restrict__ Vinv,
                                               const double* __restrict__ G, int first_order,
                                               double* __restrict__ dQ) {
    __shared__ double Y[64];
    const int i = blockIdx.x, t = threadIdx.x;
    if (first_order) {
        if (t < Spad) dQ[i * Spad + t] = G[i * Spad + t];
        return;
    }
    double acc = 0.0;
    if (t < Spad)
        for (int k = 0; k < S; ++k) acc += Vinv[k * Spad + i] * G[k * Spad + t];
    Y[t] = acc;
    __syncthreads();
    if (t >= Spad) return;
    double d = 0.0;
    if (i < S && t < S)
        for (int l = 0; l < S; ++l) d += Y[l] * V[t * Spad + l];
    dQ[i * Spad + t] = d;
}

// Every substitution parameter from D = dlogL/dQ: <D, dQ/dtheta_k> for the
// stored derivative matrices (fixed-order block sums), and the closed forms
// of the general reversible model's exchangeabilities and of the
// random-effect pairs, which need <D, Q>.
__global__ void __launch_bounds__(256) k_adj_params(int S, int Spad, const double* __restrict__ D,
                                                    const double* __restrict__ Q,
                                                    const double* __restrict__ pi,
                                                    const double* __restrict__ dQk, int n_dq,
                                                    const int* __restrict__ pairs, int n_pairs,
                                                    int n_exch, const double* __restrict__ mu,
                                                    double* __restrict__ theta) {
    const int SS = Spad * Spad;
    __shared__ double red[256];
    __shared__ double gq;
    const int t = threadIdx.x, nt = blockDim.x;
    // <D, M> for M = dQ/dtheta_k (k < n_dq), then M = Q
    for (int k = 0; k <= n_dq; ++k) {
        const double* Mk = (k < n_dq) ? dQk + (size_t)k * SS : Q;
        double acc = 0.0;
        for (int idx = t; idx < SS; idx += nt) acc += D[idx] * Mk[idx];
        red[t] = acc;
        __syncthreads();
        for (int w = nt / 2; w > 0; w >>= 1) {
            if (t < w) red[t] += red[t + w];
            __syncthreads();
        }
        if (t == 0) {
            if (k < n_dq) theta[k] = red[0];
            else gq = red[0];
        }
        __syncthreads();
    }
    // general reversible model, exchangeability E_ab (a != b; s_ab = s_ba =
    // (E_ab + E_ba) / 2, normaliser mu of the unnormalised rates):
    //   dlogL/dE_ab = [pi_b (dQ_ab - dQ_aa) + pi_a (dQ_ba - dQ_bb)] / (2 mu)
    //                 - pi_a pi_b <dQ, Q> / mu
    for (int k = t; k < n_exch; k += nt) {
        const int i = k / S, j = k % S;
        theta[k] = (i == j) ? 0.0
                            : (pi[j] * (D[i * Spad + j] - D[i * Spad + i]) +
                               pi[i] * (D[j * Spad + i] - D[j * Spad + j])) / (2.0 * mu[0]) -
                                  pi[i] * pi[j] * gq / mu[0];
    }
    for (int k = t; k < n_pairs; k += nt) {
        const int i = pairs[2 * k], j = pairs[2 * k + 1];
        const double qij = Q[i * Spad + j], qji = Q[j * Spad + i];
        theta[n_dq + k] = qij * (D[i * Spad + j] - D[i * Spad + i]) +
                          qji * (D[j * Spad + i] - D[j * Spad + j]) -
                          (pi[i] * qij + pi[j] * qji) * gq;
    }
}

int launch_adj_params(Instance* I, int model, const double* d_G, bool first_order, double* d_dQ,
                      double* d_theta) {
    ModelDev& M = I->models[model];
    const int n_pairs = M.kind == TL_MODEL_GY94RE ? TL_GY94_PAIRS : 0;
    const int n_exch = M.kind == TL_MODEL_REV ? I->S * I->S : 0;
    k_adj_dq<<<I->Spad, 64, 0, I->stream>>>(I->S, I->Spad, M.V, M.Vinv, d_G, first_order, d_dQ);
    k_adj_params<<<1, 256, 0, I->stream>>>(I->S, I->Spad, d_dQ, M.Q, M.pi, M.dQ, M.n_dq, M.pairs,
                                           n_pairs, n_exch, M.mu, d_theta);
    I->launches += 2;
    return cuda_check(I, cudaGetLastError(), "adjoint parameters");
}

}  // namespace tl
