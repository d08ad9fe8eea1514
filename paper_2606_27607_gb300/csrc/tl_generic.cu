// FP64 kernels for any state count S <= 64: the plain, one-op-per-launch
// correctness path (used for codon models in FP64 and for state counts the
// specialised kernels do not cover).
//
// A block owns kPT patterns; thread (r, i) owns state i of category r for
// all of them. Child partials of the block's patterns are staged in shared
// memory and broadcast; P is read in its transposed layout W[j][i] = P[i][j]
// so that threads i read consecutive addresses. Per-pattern maxima and the
// likelihood sums are block reductions in a fixed order.
#include <cmath>

#include "tl_internal.cuh"

namespace tl {

constexpr int kPT = 8;  // patterns per block

struct GenArgs {
    double* const* buf;
    int* const* scale;
    const int8_t* const* tipst;
    const double* W;      // [mat][R][Spad+1][Spad]
    const double* M64;    // [mat][R][Spad][Spad]
    const double* patw;
    int n_tips, P, Ppad, R, S, Spad, rescale;
    size_t wstride;       // doubles per matrix slot in W
    double catw[kMaxCat];
    double rates[kMaxCat];
};

__device__ __forceinline__ int gen_frexp(double m) {
    int E = (int)((__double_as_longlong(m) >> 52) & 0x7ff);
    if (E == 0) {
        if (m == 0.0) return 0;
        E = (int)((__double_as_longlong(m * 18446744073709551616.0) >> 52) & 0x7ff) - 64;
    }
    return E - 1022;
}
__device__ __forceinline__ double gen_scale(double x, int k) {
    if (k >= -1022 && k <= 1022) return x * __longlong_as_double((long long)(k + 1023) << 52);
    int k1 = k / 2;
    return x * __longlong_as_double((long long)(k1 + 1023) << 52) *
           __longlong_as_double((long long)(k - k1 + 1023) << 52);
}

// Block-wide reduction of kPT values per thread (op: 0 sum, 1 max); result
// broadcast through `out`.
__device__ void block_reduce_pt(double* v, double* red, double* out, int op) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int pp = 0; pp < kPT; ++pp) {
        double x = v[pp];
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = op ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[pp * 32 + warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < kPT) {
        double x = red[threadIdx.x * 32];
        for (int w = 1; w < nw; ++w) x = op ? fmax(x, red[threadIdx.x * 32 + w]) : x + red[threadIdx.x * 32 + w];
        out[threadIdx.x] = x;
    }
    __syncthreads();
}

// Load a child's contribution v[pp] = (P_c p_c)[r, p0+pp, i] for this thread.
__device__ void child_product(const GenArgs& a, int ch, const double* Wc, int r, int i, bool act,
                              int p0, double* xs, int* cum, double* v) {
    const int S = a.S, Spad = a.Spad, R = a.R;
    const int8_t* ts = (ch < a.n_tips) ? a.tipst[ch] : nullptr;
    if (ts != nullptr) {
#pragma unroll
        for (int pp = 0; pp < kPT; ++pp) {
            int s = ts[p0 + pp];
            int col = (s >= 0 && s < S) ? s : Spad;
            v[pp] = act ? Wc[((size_t)r * (Spad + 1) + col) * Spad + i] : 0.0;
        }
        return;
    }
    // stage [R][kPT][Spad] of the child
    const double* b = a.buf[ch];
    for (int idx = threadIdx.x; idx < R * kPT * Spad; idx += blockDim.x) {
        int rr = idx / (kPT * Spad), rem = idx % (kPT * Spad);
        xs[idx] = b[((size_t)rr * a.Ppad + p0) * Spad + rem];
    }
    const int* sc = a.scale[ch];
    if (sc != nullptr && threadIdx.x < kPT) cum[threadIdx.x] += sc[p0 + threadIdx.x];
    __syncthreads();
#pragma unroll
    for (int pp = 0; pp < kPT; ++pp) v[pp] = 0.0;
    if (act) {
        const double* w = Wc + (size_t)r * (Spad + 1) * Spad + i;
        const double* x = xs + (size_t)r * kPT * Spad;
        for (int j = 0; j < S; ++j) {
            double wj = w[(size_t)j * Spad];
#pragma unroll
            for (int pp = 0; pp < kPT; ++pp) v[pp] += wj * x[pp * Spad + j];
        }
    }
    __syncthreads();
}

__global__ void k_post_gen(int dest, int c0, int m0, int c1, int m1, GenArgs a) {
    extern __shared__ double sm_gen[];
    double* xs = sm_gen;                                  // R*kPT*Spad
    double* red = xs + (size_t)a.R * kPT * a.Spad;        // kPT*32
    double* bc = red + kPT * 32;                          // kPT
    __shared__ int cum[kPT];
    const int p0 = blockIdx.x * kPT;
    const int t = threadIdx.x;
    const bool act = t < a.R * a.Spad;
    const int r = act ? t / a.Spad : 0, i = act ? t % a.Spad : 0;
    if (t < kPT) cum[t] = 0;
    __syncthreads();
    double v0[kPT], v1[kPT];
    child_product(a, c0, a.W + (size_t)m0 * a.wstride, r, i, act, p0, xs, cum, v0);
    child_product(a, c1, a.W + (size_t)m1 * a.wstride, r, i, act, p0, xs, cum, v1);
    double o[kPT];
#pragma unroll
    for (int pp = 0; pp < kPT; ++pp) o[pp] = act ? v0[pp] * v1[pp] : 0.0;
    if (a.rescale) {
        block_reduce_pt(o, red, bc, 1);
        if (t < kPT) {
            int e = gen_frexp(bc[t]);
            cum[t] += e;
            bc[t] = (double)e;
        }
        __syncthreads();
#pragma unroll
        for (int pp = 0; pp < kPT; ++pp) {
            int e = (int)bc[pp];
            if (e != 0) o[pp] = gen_scale(o[pp], -e);
        }
    }
    if (act) {
        double* d = a.buf[dest];
#pragma unroll
        for (int pp = 0; pp < kPT; ++pp) d[((size_t)r * a.Ppad + p0 + pp) * a.Spad + i] = o[pp];
    }
    if (t < kPT) a.scale[dest][p0 + t] = cum[t];
}

__global__ void k_root_gen(int root, GenArgs a, const double* __restrict__ pi,
                           double* __restrict__ site, double* __restrict__ part,
                           int* __restrict__ err) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (p < a.Ppad) {
        double L = 0.0;
        int cum = 0;
        const int8_t* ts = (root < a.n_tips) ? a.tipst[root] : nullptr;
        if (ts) {
            int s = ts[p];
            double tot = 0, cw = 0;
            for (int q = 0; q < a.S; ++q) tot += pi[q];
            for (int r = 0; r < a.R; ++r) cw += a.catw[r];
            L = cw * ((s >= 0 && s < a.S) ? pi[s] : tot);
        } else {
            const double* b = a.buf[root];
            for (int r = 0; r < a.R; ++r) {
                double s = 0;
                const double* x = b + ((size_t)r * a.Ppad + p) * a.Spad;
                for (int q = 0; q < a.S; ++q) s += pi[q] * x[q];
                L += a.catw[r] * s;
            }
            if (a.scale[root]) cum = a.scale[root][p];
        }
        double l = log(L) + 0.69314718055994530942 * (double)cum;
        if (p < a.P) {
            if (!(L > 0.0) || !isfinite(l)) atomicOr(err, 1);
            if (site) site[p] = l;
            contrib = a.patw[p] * l;
        }
    }
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    __shared__ double wsum[32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = contrib;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w];
        part[blockIdx.x] = s;
    }
}

// One pre-order parent op: q_c = P_c^T (q_n o P_s p_s), gradient partials.
__global__ void k_pre_gen(tl_pre_op op, int q_in, const double* __restrict__ pi, GenArgs a,
                          double* q_out0, double* q_out1, double* __restrict__ gpart, int n_parts) {
    extern __shared__ double sm_gen[];
    const int R = a.R, Spad = a.Spad, S = a.S;
    const size_t tileN = (size_t)R * kPT * Spad;
    double* xs = sm_gen;            // staging
    double* us = xs + tileN;        // u_c for the transposed product
    double* red = us + tileN;       // kPT*32
    double* bc = red + kPT * 32;    // kPT
    double* den = bc + kPT;         // kPT
    __shared__ int cum[kPT];
    const int p0 = blockIdx.x * kPT;
    const int t = threadIdx.x;
    const bool act = t < R * Spad;
    const int r = act ? t / Spad : 0, i = act ? t % Spad : 0;
    if (t < kPT) cum[t] = 0;
    __syncthreads();
    double q[kPT];
#pragma unroll
    for (int pp = 0; pp < kPT; ++pp) {
        if (!act) q[pp] = 0.0;
        else if (q_in < 0) q[pp] = pi[i];
        else q[pp] = a.buf[q_in][((size_t)r * a.Ppad + p0 + pp) * Spad + i];
    }
    double v[2][kPT], d[2][kPT];
    for (int c = 0; c < 2; ++c) {
        child_product(a, op.child[c], a.W + (size_t)op.mat[c] * a.wstride, r, i, act, p0, xs, cum,
                      v[c]);
        if (op.dmat[c] >= 0)
            child_product(a, op.child[c], a.W + (size_t)op.dmat[c] * a.wstride, r, i, act, p0, xs,
                          cum, d[c]);
        else
            for (int pp = 0; pp < kPT; ++pp) d[c][pp] = 0.0;
    }
    double tmp[kPT];
#pragma unroll
    for (int pp = 0; pp < kPT; ++pp) tmp[pp] = act ? a.catw[r] * q[pp] * v[0][pp] * v[1][pp] : 0.0;
    block_reduce_pt(tmp, red, bc, 0);
    if (t < kPT) den[t] = bc[t];
    __syncthreads();
    for (int c = 0; c < 2; ++c) {
        double u[kPT];
#pragma unroll
        for (int pp = 0; pp < kPT; ++pp) u[pp] = q[pp] * v[1 - c][pp];
        if (op.edge[c] >= 0) {
#pragma unroll
            for (int pp = 0; pp < kPT; ++pp) tmp[pp] = act ? a.catw[r] * u[pp] * d[c][pp] : 0.0;
            block_reduce_pt(tmp, red, bc, 0);
            if (t == 0) {
                double g = 0;
                for (int pp = 0; pp < kPT; ++pp)
                    if (p0 + pp < a.P) g += a.patw[p0 + pp] * (bc[pp] / den[pp]);
                gpart[(size_t)op.edge[c] * n_parts + blockIdx.x] = g;
            }
            __syncthreads();
        }
        double* qo = c == 0 ? q_out0 : q_out1;
        if (qo != nullptr) {
            if (act)
                for (int pp = 0; pp < kPT; ++pp) us[((size_t)r * kPT + pp) * Spad + i] = u[pp];
            __syncthreads();
            // q_c[j] = sum_i P[i][j] u[i]; thread (r, j=i)
            double qc[kPT];
#pragma unroll
            for (int pp = 0; pp < kPT; ++pp) qc[pp] = 0.0;
            if (act && i < S) {
                const double* Pm = a.M64 + (size_t)op.mat[c] * R * Spad * Spad + (size_t)r * Spad * Spad;
                for (int ii = 0; ii < S; ++ii) {
                    double pij = Pm[(size_t)ii * Spad + i];
#pragma unroll
                    for (int pp = 0; pp < kPT; ++pp) qc[pp] += pij * us[((size_t)r * kPT + pp) * Spad + ii];
                }
            }
            block_reduce_pt(qc, red, bc, 1);
#pragma unroll
            for (int pp = 0; pp < kPT; ++pp) {
                int e = gen_frexp(bc[pp]);
                if (e != 0) qc[pp] = gen_scale(qc[pp], -e);
            }
            if (act)
                for (int pp = 0; pp < kPT; ++pp) qo[((size_t)r * a.Ppad + p0 + pp) * Spad + i] = qc[pp];
            __syncthreads();
        }
    }
}

__global__ void k_edge_gen(tl_edge e, const double* __restrict__ Q, GenArgs a,
                           double* __restrict__ gpart, int n_parts) {
    extern __shared__ double sm_gen[];
    const int R = a.R, Spad = a.Spad, S = a.S;
    double* xs = sm_gen;
    double* red = xs + (size_t)R * kPT * Spad;
    double* bc = red + kPT * 32;
    double* den = bc + kPT;
    const int p0 = blockIdx.x * kPT;
    const int t = threadIdx.x;
    const bool act = t < R * Spad;
    const int r = act ? t / Spad : 0, i = act ? t % Spad : 0;
    const int8_t* ts = (e.post < a.n_tips) ? a.tipst[e.post] : nullptr;
    // stage p_c as [R][kPT][Spad]
    for (int idx = t; idx < R * kPT * Spad; idx += blockDim.x) {
        int rr = idx / (kPT * Spad), rem = idx % (kPT * Spad);
        int pp = rem / Spad, j = rem % Spad;
        double x;
        if (ts) {
            int s = ts[p0 + pp];
            x = (j < S) ? ((s >= 0 && s < S) ? (double)(s == j) : 1.0) : 0.0;
        } else {
            x = a.buf[e.post][((size_t)rr * a.Ppad + p0) * Spad + rem];
        }
        xs[idx] = x;
    }
    __syncthreads();
    double num[kPT], dn[kPT];
    const double* qb = a.buf[e.pre];
#pragma unroll
    for (int pp = 0; pp < kPT; ++pp) {
        num[pp] = 0.0;
        dn[pp] = 0.0;
        if (act && i < S) {
            double qi = qb[((size_t)r * a.Ppad + p0 + pp) * Spad + i];
            const double* x = xs + ((size_t)r * kPT + pp) * Spad;
            double qx = 0;
            for (int j = 0; j < S; ++j) qx += Q[(size_t)i * Spad + j] * x[j];
            num[pp] = a.catw[r] * a.rates[r] * qi * qx;
            dn[pp] = a.catw[r] * qi * x[i];
        }
    }
    block_reduce_pt(dn, red, bc, 0);
    if (t < kPT) den[t] = bc[t];
    __syncthreads();
    block_reduce_pt(num, red, bc, 0);
    if (t == 0) {
        double g = 0;
        for (int pp = 0; pp < kPT; ++pp)
            if (p0 + pp < a.P) g += a.patw[p0 + pp] * (bc[pp] / den[pp]);
        gpart[(size_t)e.edge * n_parts + blockIdx.x] = g;
    }
}

static GenArgs gen_args(const Instance* I) {
    GenArgs a;
    a.buf = reinterpret_cast<double* const*>(I->d_buf);
    a.scale = I->d_scale;
    a.tipst = I->d_tipst;
    a.W = reinterpret_cast<const double*>(I->d_matw);
    a.M64 = I->d_mat64;
    a.patw = I->d_patw;
    a.n_tips = I->n_tips;
    a.P = I->P;
    a.Ppad = I->Ppad;
    a.R = I->R;
    a.S = I->S;
    a.Spad = I->Spad;
    a.rescale = I->rescale;
    a.wstride = I->matw_stride;
    for (int r = 0; r < kMaxCat; ++r) {
        a.catw[r] = r < I->R ? I->h_catw[r] : 0.0;
        a.rates[r] = r < I->R ? I->h_rates[r] : 0.0;
    }
    return a;
}

static int gen_threads(const Instance* I) { return ((I->R * I->Spad + 31) / 32) * 32; }

// ---- on-the-fly transition matrices -----------------------------------------
// For a large state space with a single site pattern no transition matrix is
// reused, so forming P(t) (S^3 per edge and category) costs more than the
// pruning itself (Sec. "Discussion"). Here a child's product is taken in the
// eigenbasis: v = V (e^{lambda rho_r t_c} o (V^-1 p_c)), two S^2 products per
// pattern. A block per op (the ops of one tree level per launch), thread
// (category r, state i); V and V^-1 in shared memory. Rescaling and the
// cumulative exponents are those of the generic post-order kernel; padding
// patterns get all-ones partials and exponent 0.
__global__ void k_post_eig(const EigOp* __restrict__ ops, GenArgs a, const double* __restrict__ V,
                           const double* __restrict__ Vinv, const double* __restrict__ lam) {
    extern __shared__ double sm_eig[];
    const int S = a.S, Spad = a.Spad, R = a.R;
    const int SS = Spad * Spad;
    double* Vs = sm_eig;              // [Spad][Spad]
    double* Vi = Vs + SS;             // [Spad][Spad]
    double* ex = Vi + SS;             // [2][R][Spad] e^{lambda rho t}
    double* xs = ex + 2 * R * Spad;   // [R][Spad] child partial of this pattern
    double* ws = xs + R * Spad;       // [R][Spad] V^-1 p, scaled
    __shared__ double red[32];
    const EigOp op = ops[blockIdx.x];
    const int t = threadIdx.x, nt = blockDim.x;
    const bool act = t < R * Spad;
    const int r = act ? t / Spad : 0, i = act ? t % Spad : 0;
    for (int idx = t; idx < SS; idx += nt) {
        Vs[idx] = V[idx];
        Vi[idx] = Vinv[idx];
    }
    for (int idx = t; idx < 2 * R * Spad; idx += nt) {
        const int c = idx / (R * Spad), rr = (idx / Spad) % R, k = idx % Spad;
        ex[idx] = k < S ? exp(lam[k] * a.rates[rr] * op.len[c]) : 0.0;
    }
    double* dst = a.buf[op.dest];
    for (int p = 0; p < a.Ppad; ++p) {
        if (p >= a.P) {  // padding
            if (act) dst[((size_t)r * a.Ppad + p) * Spad + i] = i < S ? 1.0 : 0.0;
            if (t == 0) a.scale[op.dest][p] = 0;
            continue;
        }
        double prod = 1.0;
        int cum = 0;
        for (int c = 0; c < 2; ++c) {
            const int ch = op.child[c];
            __syncthreads();  // xs, ws free
            const int8_t* ts = ch < a.n_tips ? a.tipst[ch] : nullptr;
            if (act) {
                double x = 0.0;
                if (i < S) {
                    if (ts) {
                        const int s = ts[p];
                        x = (s < 0 || s >= S || s == i) ? 1.0 : 0.0;
                    } else {
                        x = a.buf[ch][((size_t)r * a.Ppad + p) * Spad + i];
                    }
                }
                xs[t] = x;
            }
            if (!ts && a.scale[ch]) cum += a.scale[ch][p];
            __syncthreads();
            if (act) {
                double w = 0.0;
                if (i < S)
                    for (int j = 0; j < S; ++j) w += Vi[i * Spad + j] * xs[r * Spad + j];
                ws[t] = w * ex[(c * R + r) * Spad + i];
            }
            __syncthreads();
            double v = 0.0;
            if (act && i < S)
                for (int k = 0; k < S; ++k) v += Vs[i * Spad + k] * ws[r * Spad + k];
            prod *= v;
        }
        if (!act || i >= S) prod = 0.0;
        int e = 0;
        if (a.rescale) {
            double m = prod;
            for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((t & 31) == 0) red[t >> 5] = m;
            __syncthreads();
            m = red[0];
            for (int w = 1; w < (nt >> 5); ++w) m = fmax(m, red[w]);
            e = gen_frexp(m);
            __syncthreads();  // red read by every thread before the next pattern
        }
        if (act) dst[((size_t)r * a.Ppad + p) * Spad + i] = e ? gen_scale(prod, -e) : prod;
        if (t == 0) a.scale[op.dest][p] = cum + e;
    }
}

int launch_post_eig(Instance* I, int model, const EigOp* d_ops, const int* level_start,
                    int n_levels) {
    GenArgs a = gen_args(I);
    const ModelDev& M = I->models[model];
    const size_t smem = (2 * (size_t)I->Spad * I->Spad + 4 * (size_t)I->R * I->Spad) * sizeof(double);
    cudaFuncSetAttribute(k_post_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int L = 0; L < n_levels; ++L) {
        const int n = level_start[L + 1] - level_start[L];
        if (n <= 0) continue;
        k_post_eig<<<n, gen_threads(I), smem, I->stream>>>(d_ops + level_start[L], a, M.V, M.Vinv,
                                                          M.lam);
        I->launches += 1;
    }
    return cuda_check(I, cudaGetLastError(), "on-the-fly post-order kernel");
}

int generic_parts(const Instance* I) { return I->Ppad / kPT; }

int launch_post_generic(Instance* I, const tl_op* ops, int n_ops) {
    GenArgs a = gen_args(I);
    size_t smem = ((size_t)I->R * kPT * I->Spad + kPT * 32 + kPT) * sizeof(double);
    cudaFuncSetAttribute(k_post_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int k = 0; k < n_ops; ++k) {
        const tl_op& o = ops[k];
        k_post_gen<<<I->Ppad / kPT, gen_threads(I), smem, I->stream>>>(o.dest, o.child1, o.mat1,
                                                                       o.child2, o.mat2, a);
    }
    I->launches += n_ops;
    return cuda_check(I, cudaGetLastError(), "generic post-order kernel");
}

int launch_root_generic(Instance* I, int root, int model, double* d_site, double* d_part,
                        int n_parts) {
    (void)n_parts;
    GenArgs a = gen_args(I);
    int blocks = (I->Ppad + 127) / 128;
    k_root_gen<<<blocks, 128, 0, I->stream>>>(root, a, I->models[model].pi, d_site, d_part,
                                              I->d_err + 1);
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "generic root kernel");
}

int launch_pre_generic(Instance* I, const tl_pre_op* ops, int n_ops, int model, double* d_gpart,
                       int n_parts) {
    GenArgs a = gen_args(I);
    size_t tileN = (size_t)I->R * kPT * I->Spad;
    size_t smem = (2 * tileN + kPT * 32 + 2 * kPT) * sizeof(double);
    cudaFuncSetAttribute(k_pre_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int k = 0; k < n_ops; ++k) {
        const tl_pre_op& o = ops[k];
        double* q0 = o.pre[0] >= 0 ? reinterpret_cast<double*>(I->h_buf[o.pre[0]]) : nullptr;
        double* q1 = o.pre[1] >= 0 ? reinterpret_cast<double*>(I->h_buf[o.pre[1]]) : nullptr;
        k_pre_gen<<<I->Ppad / kPT, gen_threads(I), smem, I->stream>>>(
            o, o.parent_pre, I->models[model].pi, a, q0, q1, d_gpart, n_parts);
    }
    I->launches += n_ops;
    return cuda_check(I, cudaGetLastError(), "generic pre-order kernel");
}

int launch_edge_generic(Instance* I, const tl_edge* edges, int n_edges, int model,
                        double* d_gpart, int n_parts) {
    GenArgs a = gen_args(I);
    size_t smem = ((size_t)I->R * kPT * I->Spad + kPT * 32 + 2 * kPT) * sizeof(double);
    cudaFuncSetAttribute(k_edge_gen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int k = 0; k < n_edges; ++k)
        k_edge_gen<<<I->Ppad / kPT, gen_threads(I), smem, I->stream>>>(
            edges[k], I->models[model].Q, a, d_gpart, n_parts);
    I->launches += n_edges;
    return cuda_check(I, cudaGetLastError(), "generic edge kernel");
}

}  // namespace tl
