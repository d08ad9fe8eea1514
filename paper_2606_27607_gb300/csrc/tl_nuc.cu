// Four-state (nucleotide) kernels: post-order pruning with per-pattern
// power-of-two rescaling, root log-likelihood, fused pre-order pass with
// branch-length gradient, and edge derivatives from stored partials.
//
// Design: patterns are independent given the tree (Sec. "Benchmarks on
// NVIDIA and AMD GPUs": the alignment splits into conditionally independent
// blocks), so one warp owns a tile of 32 patterns -- one lane per pattern,
// all rate categories in registers -- and walks the WHOLE operation list for
// its tile in a single launch. No warp ever waits for another. A child that
// an earlier op of the same list produced is read from a warp-private
// shared-memory slot (the host assigns slots); only results the caller asked
// for go to HBM. Partials are [category][pattern][4] so each lane's float4 /
// double2x2 accesses coalesce across the warp. Matrices are read through the
// read-only path with warp-uniform addresses (one broadcast per load).
// A tip with states uses a column of P (or the row sums for an ambiguous
// code) instead of a product (the benchmark spec: tip-state lookups).
#include <cmath>

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

// P x with P given by its columns c0..c3: x0 c0 + x1 c1 + x2 c2 + x3 c3.
template <typename T>
__device__ __forceinline__ V4<T> matvec(const T* col, V4<T> x) {
    V4<T> c0 = ldg4(col), c1 = ldg4(col + 4), c2 = ldg4(col + 8), c3 = ldg4(col + 12);
    V4<T> r;
    r.x = x.x * c0.x + x.y * c1.x + x.z * c2.x + x.w * c3.x;
    r.y = x.x * c0.y + x.y * c1.y + x.z * c2.y + x.w * c3.y;
    r.z = x.x * c0.z + x.y * c1.z + x.z * c2.z + x.w * c3.z;
    r.w = x.x * c0.w + x.y * c1.w + x.z * c2.w + x.w * c3.w;
    return r;
}
// P^T u: component j is column j . u
template <typename T>
__device__ __forceinline__ V4<T> matTvec(const T* col, V4<T> u) {
    V4<T> c0 = ldg4(col), c1 = ldg4(col + 4), c2 = ldg4(col + 8), c3 = ldg4(col + 12);
    return {dot(c0, u), dot(c1, u), dot(c2, u), dot(c3, u)};
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

__device__ __forceinline__ int tip_col(int8_t s) { return (s >= 0 && s < 4) ? (int)s : 4; }

// ---------------------------------------------------------------------------
// post-order
// ---------------------------------------------------------------------------
template <typename T, int RM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_post4(const DevPostOp* __restrict__ ops, int n_ops, PathArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kWarpsPerBlock + warp;
    if (tile * kTile >= a.Ppad) return;
    const int p = tile * kTile + lane;
    const int R = a.R;
    V4<T>* slots = reinterpret_cast<V4<T>*>(smem_raw) + (size_t)warp * a.n_slots * RM * 32;
    int* sexp = reinterpret_cast<int*>(reinterpret_cast<V4<T>*>(smem_raw) +
                                       (size_t)kWarpsPerBlock * a.n_slots * RM * 32) +
                warp * a.n_slots * 32;

    for (int k = 0; k < n_ops; ++k) {
        const DevPostOp op = ops[k];
        V4<T> acc[RM];
        int cum = 0;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int ch = op.child[c];
            const T* mc = a.mat + (size_t)op.mat[c] * a.mat_stride;
            const int8_t* ts = (ch < a.n_tips) ? a.tipst[ch] : nullptr;
            if (ts != nullptr) {
                const int col = tip_col(__ldg(ts + p));
#pragma unroll
                for (int r = 0; r < RM; ++r) {
                    if (r < R) {
                        V4<T> v = ldg4(mc + (r * kColStride + col) * 4);
                        acc[r] = (c == 0) ? v : mul(acc[r], v);
                    }
                }
            } else {
                V4<T> x[RM];
                if (op.slot_in[c] >= 0) {
                    const V4<T>* s = slots + (size_t)op.slot_in[c] * RM * 32;
#pragma unroll
                    for (int r = 0; r < RM; ++r)
                        if (r < R) x[r] = s[r * 32 + lane];
                    cum += sexp[op.slot_in[c] * 32 + lane];
                } else {
                    const T* b = a.buf[ch];
#pragma unroll
                    for (int r = 0; r < RM; ++r)
                        if (r < R) x[r] = ld4(b + ((size_t)r * a.Ppad + p) * 4);
                    const int* sc = a.scale[ch];
                    if (sc != nullptr) cum += sc[p];
                }
#pragma unroll
                for (int r = 0; r < RM; ++r) {
                    if (r < R) {
                        V4<T> v = matvec(mc + r * kColStride * 4, x[r]);
                        acc[r] = (c == 0) ? v : mul(acc[r], v);
                    }
                }
            }
        }
        if (a.rescale) {
            T m = T(0);
#pragma unroll
            for (int r = 0; r < RM; ++r)
                if (r < R) m = fmax(m, vmax(acc[r]));
            const int e = frexp_exp(m);
            if (e != 0) {
                scale_by_pow2(acc, R < RM ? R : RM, -e);
                cum += e;
            }
        }
        if (op.store) {
            T* d = a.buf[op.dest];
#pragma unroll
            for (int r = 0; r < RM; ++r)
                if (r < R) st4(d + ((size_t)r * a.Ppad + p) * 4, acc[r]);
            a.scale[op.dest][p] = cum;
        }
        if (op.slot_out >= 0) {
            V4<T>* s = slots + (size_t)op.slot_out * RM * 32;
#pragma unroll
            for (int r = 0; r < RM; ++r)
                if (r < R) s[r * 32 + lane] = acc[r];
            sexp[op.slot_out * 32 + lane] = cum;
        }
    }
}

// ---------------------------------------------------------------------------
// root log-likelihood: per-warp partial sums of w_p l_p
// ---------------------------------------------------------------------------
template <typename T, int RM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_root4(int root, PathArgs<T> a, const double* __restrict__ pi, double* __restrict__ site,
        double* __restrict__ part, int* __restrict__ err) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kWarpsPerBlock + warp;
    if (tile * kTile >= a.Ppad) return;
    const int p = tile * kTile + lane;
    double L = 0.0;
    int cum = 0;
    const int8_t* ts = (root < a.n_tips) ? a.tipst[root] : nullptr;
    if (ts != nullptr) {
        int s = ts[p];
        double tot = 0;
        for (int q = 0; q < 4; ++q) tot += pi[q];
        L = (s >= 0 && s < 4) ? pi[s] : tot;
        double cw = 0;
        for (int r = 0; r < a.R; ++r) cw += (double)a.catw[r];
        L *= cw;
    } else {
        const T* b = a.buf[root];
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            if (r < a.R) {
                V4<T> x = ld4(b + ((size_t)r * a.Ppad + p) * 4);
                double s = pi[0] * (double)x.x + pi[1] * (double)x.y + pi[2] * (double)x.z +
                           pi[3] * (double)x.w;
                L += (double)a.catw[r] * s;
            }
        }
        const int* sc = a.scale[root];
        if (sc) cum = sc[p];
    }
    double l = log(L) + 0.69314718055994530942 * (double)cum;
    double contrib = 0.0;
    if (p < a.P) {
        if (!(L > 0.0) || !isfinite(l)) atomicOr(err, 1);
        if (site) site[p] = l;
        contrib = a.patw[p] * l;
    }
    contrib = warp_sum(contrib);
    if (lane == 0) part[tile] = contrib;
}

// ---------------------------------------------------------------------------
// fused pre-order pass + branch-length gradient
// ---------------------------------------------------------------------------
template <typename T, int RM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_pre4(const DevPreOp* __restrict__ ops, int n_ops, PathArgs<T> a, const T* __restrict__ piw,
       double* __restrict__ gpart, int n_tiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kWarpsPerBlock + warp;
    if (tile * kTile >= a.Ppad) return;
    const int p = tile * kTile + lane;
    const int R = a.R;
    V4<T>* slots = reinterpret_cast<V4<T>*>(smem_raw) + (size_t)warp * a.n_slots * RM * 32;
    const V4<T> piv = ldg4(piw);
    const double wp = (p < a.P) ? a.patw[p] : 0.0;

    for (int k = 0; k < n_ops; ++k) {
        const DevPreOp op = ops[k];
        V4<T> q[RM];
        if (op.q_slot_in == -2) {
#pragma unroll
            for (int r = 0; r < RM; ++r) q[r] = piv;
        } else if (op.q_slot_in >= 0) {
            const V4<T>* s = slots + (size_t)op.q_slot_in * RM * 32;
#pragma unroll
            for (int r = 0; r < RM; ++r)
                if (r < R) q[r] = s[r * 32 + lane];
        } else {
            const T* b = a.buf[op.q_buf_in];
#pragma unroll
            for (int r = 0; r < RM; ++r)
                if (r < R) q[r] = ld4(b + ((size_t)r * a.Ppad + p) * 4);
        }
        // v_c = P_c p_c and d_c = dP_c p_c for both children
        V4<T> v[2][RM], d[2][RM];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int ch = op.child[c];
            const T* mc = a.mat + (size_t)op.mat[c] * a.mat_stride;
            const T* dc = (op.dmat[c] >= 0) ? a.mat + (size_t)op.dmat[c] * a.mat_stride : nullptr;
            const int8_t* ts = (ch < a.n_tips) ? a.tipst[ch] : nullptr;
            if (ts != nullptr) {
                const int col = tip_col(__ldg(ts + p));
#pragma unroll
                for (int r = 0; r < RM; ++r) {
                    if (r < R) {
                        v[c][r] = ldg4(mc + (r * kColStride + col) * 4);
                        if (dc) d[c][r] = ldg4(dc + (r * kColStride + col) * 4);
                    }
                }
            } else {
                const T* b = a.buf[ch];
#pragma unroll
                for (int r = 0; r < RM; ++r) {
                    if (r < R) {
                        V4<T> x = ld4(b + ((size_t)r * a.Ppad + p) * 4);
                        v[c][r] = matvec(mc + r * kColStride * 4, x);
                        if (dc) d[c][r] = matvec(dc + r * kColStride * 4, x);
                    }
                }
            }
        }
        // den = sum_r w_r q . (v_a o v_b): the pattern likelihood up to scale
        T den = T(0);
#pragma unroll
        for (int r = 0; r < RM; ++r)
            if (r < R) den += a.catw[r] * dot(q[r], mul(v[0][r], v[1][r]));
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            V4<T> u[RM];
#pragma unroll
            for (int r = 0; r < RM; ++r)
                if (r < R) u[r] = mul(q[r], v[1 - c][r]);
            if (op.edge[c] >= 0) {
                T num = T(0);
#pragma unroll
                for (int r = 0; r < RM; ++r)
                    if (r < R) num += a.catw[r] * dot(u[r], d[c][r]);
                double g = (p < a.P) ? wp * ((double)num / (double)den) : 0.0;
                g = warp_sum(g);
                if (lane == 0) gpart[(size_t)op.edge[c] * n_tiles + tile] = g;
            }
            if (op.need_q[c]) {
                const T* mc = a.mat + (size_t)op.mat[c] * a.mat_stride;
                V4<T> qc[RM];
                T m = T(0);
#pragma unroll
                for (int r = 0; r < RM; ++r) {
                    if (r < R) {
                        qc[r] = matTvec(mc + r * kColStride * 4, u[r]);
                        m = fmax(m, vmax(qc[r]));
                    }
                }
                const int e = frexp_exp(m);
                if (e != 0) scale_by_pow2(qc, R < RM ? R : RM, -e);
                if (op.q_slot_out[c] >= 0) {
                    V4<T>* s = slots + (size_t)op.q_slot_out[c] * RM * 32;
#pragma unroll
                    for (int r = 0; r < RM; ++r)
                        if (r < R) s[r * 32 + lane] = qc[r];
                }
                if (op.q_buf_out[c] >= 0) {
                    T* b = a.buf[op.q_buf_out[c]];
#pragma unroll
                    for (int r = 0; r < RM; ++r)
                        if (r < R) st4(b + ((size_t)r * a.Ppad + p) * 4, qc[r]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// edge derivatives from stored pre- and post-order partials
// ---------------------------------------------------------------------------
template <typename T, int RM>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_edge4(const DevEdge* __restrict__ edges, int n_edges, PathArgs<T> a, const T* __restrict__ Qw,
        double* __restrict__ gpart, int n_tiles) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kWarpsPerBlock + warp;
    if (tile * kTile >= a.Ppad) return;
    const int p = tile * kTile + lane;
    const int R = a.R;
    // Q rows as V4
    const V4<T> q0 = ldg4(Qw), q1 = ldg4(Qw + 4), q2 = ldg4(Qw + 8), q3 = ldg4(Qw + 12);
    const double wp = (p < a.P) ? a.patw[p] : 0.0;
    for (int k = 0; k < n_edges; ++k) {
        const DevEdge e = edges[k];
        const int8_t* ts = (e.post < a.n_tips) ? a.tipst[e.post] : nullptr;
        const T* qb = a.buf[e.pre];
        T num = T(0), den = T(0);
        V4<T> onehot;
        if (ts) {
            int s = ts[p];
            bool amb = !(s >= 0 && s < 4);
            onehot = {T(amb || s == 0), T(amb || s == 1), T(amb || s == 2), T(amb || s == 3)};
        }
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            if (r < R) {
                V4<T> x = ts ? onehot : ld4(a.buf[e.post] + ((size_t)r * a.Ppad + p) * 4);
                V4<T> qq = ld4(qb + ((size_t)r * a.Ppad + p) * 4);
                V4<T> Qx = {dot(q0, x), dot(q1, x), dot(q2, x), dot(q3, x)};
                num += a.catw[r] * a.rates[r] * dot(qq, Qx);
                den += a.catw[r] * dot(qq, x);
            }
        }
        double g = (p < a.P) ? wp * ((double)num / (double)den) : 0.0;
        g = warp_sum(g);
        if (lane == 0) gpart[(size_t)e.edge * n_tiles + tile] = g;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
static PathArgs<T> make_args(const Instance* I, int n_slots) {
    PathArgs<T> a;
    a.buf = reinterpret_cast<T* const*>(I->d_buf);
    a.scale = I->d_scale;
    a.tipst = I->d_tipst;
    a.mat = reinterpret_cast<const T*>(I->d_matw);
    a.patw = I->d_patw;
    a.n_tips = I->n_tips;
    a.P = I->P;
    a.Ppad = I->Ppad;
    a.R = I->R;
    a.S = I->S;
    a.Spad = I->Spad;
    a.n_slots = n_slots;
    a.rescale = I->rescale;
    a.mat_stride = (int)I->matw_stride;
    for (int r = 0; r < kMaxCat; ++r) {
        a.catw[r] = (T)(r < I->R ? I->h_catw[r] : 0.0);
        a.rates[r] = (T)(r < I->R ? I->h_rates[r] : 0.0);
    }
    return a;
}

int nuc_smem_per_slot(const Instance* I) {
    const int RM = I->R <= 4 ? 4 : 8;
    return RM * 32 * 4 * I->elt + 32 * (int)sizeof(int);
}

static int n_blocks(const Instance* I) {
    const int tiles = I->Ppad / kTile;
    return (tiles + kWarpsPerBlock - 1) / kWarpsPerBlock;
}

template <typename T, int RM>
static void post4_t(Instance* I, const DevPostOp* d_ops, int n_ops, int n_slots) {
    size_t smem = (size_t)kWarpsPerBlock * n_slots * (RM * 32 * sizeof(V4<T>) + 32 * sizeof(int));
    cudaFuncSetAttribute(k_post4<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_post4<T, RM><<<n_blocks(I), kWarpsPerBlock * 32, smem, I->stream>>>(d_ops, n_ops,
                                                                           make_args<T>(I, n_slots));
}

int launch_post4(Instance* I, const DevPostOp* d_ops, int n_ops, int n_slots) {
    if (I->prec == kF32) {
        if (I->R <= 4) post4_t<float, 4>(I, d_ops, n_ops, n_slots);
        else post4_t<float, 8>(I, d_ops, n_ops, n_slots);
    } else {
        if (I->R <= 4) post4_t<double, 4>(I, d_ops, n_ops, n_slots);
        else post4_t<double, 8>(I, d_ops, n_ops, n_slots);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "post-order kernel");
}

int launch_root4(Instance* I, int root, int model, double* d_site, double* d_part, int n_tiles) {
    (void)n_tiles;
    const double* pi = I->models[model].pi;
    if (I->prec == kF32) {
        if (I->R <= 4)
            k_root4<float, 4><<<n_blocks(I), kWarpsPerBlock * 32, 0, I->stream>>>(
                root, make_args<float>(I, 0), pi, d_site, d_part, I->d_err + 1);
        else
            k_root4<float, 8><<<n_blocks(I), kWarpsPerBlock * 32, 0, I->stream>>>(
                root, make_args<float>(I, 0), pi, d_site, d_part, I->d_err + 1);
    } else {
        if (I->R <= 4)
            k_root4<double, 4><<<n_blocks(I), kWarpsPerBlock * 32, 0, I->stream>>>(
                root, make_args<double>(I, 0), pi, d_site, d_part, I->d_err + 1);
        else
            k_root4<double, 8><<<n_blocks(I), kWarpsPerBlock * 32, 0, I->stream>>>(
                root, make_args<double>(I, 0), pi, d_site, d_part, I->d_err + 1);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "root kernel");
}

template <typename T, int RM>
static void pre4_t(Instance* I, const DevPreOp* d_ops, int n_ops, int n_slots, const void* piw,
                   double* d_gpart, int n_tiles) {
    size_t smem = (size_t)kWarpsPerBlock * n_slots * RM * 32 * sizeof(V4<T>);
    cudaFuncSetAttribute(k_pre4<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pre4<T, RM><<<n_blocks(I), kWarpsPerBlock * 32, smem, I->stream>>>(
        d_ops, n_ops, make_args<T>(I, n_slots), reinterpret_cast<const T*>(piw), d_gpart, n_tiles);
}

int launch_pre4(Instance* I, const DevPreOp* d_ops, int n_ops, int n_slots, int model,
                double* d_gpart, int n_tiles) {
    const void* piw = I->models[model].piw;
    if (I->prec == kF32) {
        if (I->R <= 4) pre4_t<float, 4>(I, d_ops, n_ops, n_slots, piw, d_gpart, n_tiles);
        else pre4_t<float, 8>(I, d_ops, n_ops, n_slots, piw, d_gpart, n_tiles);
    } else {
        if (I->R <= 4) pre4_t<double, 4>(I, d_ops, n_ops, n_slots, piw, d_gpart, n_tiles);
        else pre4_t<double, 8>(I, d_ops, n_ops, n_slots, piw, d_gpart, n_tiles);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "pre-order kernel");
}

int launch_edge4(Instance* I, const DevEdge* d_edges, int n_edges, int model, double* d_gpart,
                 int n_tiles) {
    const void* Qw = I->models[model].Qw;
    if (I->prec == kF32) {
        if (I->R <= 4)
            k_edge4<float, 4><<<n_blocks(I), kWarpsPerBlock * 32, 0, I->stream>>>(
                d_edges, n_edges, make_args<float>(I, 0), (const float*)Qw, d_gpart, n_tiles);
        else
            k_edge4<float, 8><<<n_blocks(I), kWarpsPerBlock * 32, 0, I->stream>>>(
                d_edges, n_edges, make_args<float>(I, 0), (const float*)Qw, d_gpart, n_tiles);
    } else {
        if (I->R <= 4)
            k_edge4<double, 4><<<n_blocks(I), kWarpsPerBlock * 32, 0, I->stream>>>(
                d_edges, n_edges, make_args<double>(I, 0), (const double*)Qw, d_gpart, n_tiles);
        else
            k_edge4<double, 8><<<n_blocks(I), kWarpsPerBlock * 32, 0, I->stream>>>(
                d_edges, n_edges, make_args<double>(I, 0), (const double*)Qw, d_gpart, n_tiles);
    }
    I->launches += 1;
    return cuda_check(I, cudaGetLastError(), "edge-derivative kernel");
}

}  // namespace tl
