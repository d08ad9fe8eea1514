// Node-height ratio transform and its chain rule (Sec. "Algorithmic
// advances": node heights and branch-specific rates are inferred together
// by a ratio transform of the node heights that keeps every node older than
// its descendants; the branch-length gradient of the pre-order pass feeds
// it).
//
// Tips have fixed heights; internal node v other than the root has the
// anchor a_v = largest tip height below it and a ratio r_v in (0, 1):
//   h_v = a_v + r_v (h_parent(v) - a_v),   t_v = rho_v (h_parent(v) - h_v).
// Gradient from dlogL/dt = g: the height derivative of v collects
// -rho_v g_v and rho_c g_c of its children; the total derivative G_v adds
// r_c G_c of each internal child c (whose height moves with h_v), children
// first; dlogL/dr_v = (h_parent(v) - a_v) G_v, dlogL/dh_root = G_root,
// dlogL/drho_v = (h_parent(v) - h_v) g_v.
//
// One block walks the tree level by level (levels from the host, a
// __syncthreads between levels): anchors and G bottom-up, heights top-down,
// the rest elementwise.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tl_internal.cuh"

namespace tl {

struct RatioDev {
    const int* parent;     // [n]
    const int* child;      // [n_tips - 1][2]
    const int* order;      // nodes by depth, root first
    const int* level;      // [n_levels + 1] offsets into order
    const double* tip_h;   // [n_tips]
    const double* ratio;   // [n_tips - 1]
    const double* rate;    // [n]
    const double* g;       // [n] dlogL/dt (gradient mode)
    double* anc;           // [n] scratch
    double* h;             // [n] out
    double* len;           // [n] out
    double* G;             // [n] scratch
    double* g_ratio;       // [n_tips - 1] out
    double* g_rate;        // [n] out
    double* g_root;        // [1] out
    double root_h;
    int n_tips, n, n_levels, grad;
};

__global__ void __launch_bounds__(1024) k_ratio(RatioDev d) {
    const int t = threadIdx.x, nt = blockDim.x, N = d.n_tips, root = d.n - 1;
    // anchors, deepest level first
    for (int L = d.n_levels - 1; L >= 0; --L) {
        for (int k = d.level[L] + t; k < d.level[L + 1]; k += nt) {
            const int v = d.order[k];
            d.anc[v] = v < N ? d.tip_h[v]
                             : fmax(d.anc[d.child[2 * (v - N)]], d.anc[d.child[2 * (v - N) + 1]]);
        }
        __syncthreads();
    }
    // heights, root first
    for (int L = 0; L < d.n_levels; ++L) {
        for (int k = d.level[L] + t; k < d.level[L + 1]; k += nt) {
            const int v = d.order[k];
            if (v < N) d.h[v] = d.tip_h[v];
            else if (v == root) d.h[v] = d.root_h;
            else d.h[v] = d.anc[v] + d.ratio[v - N] * (d.h[d.parent[v]] - d.anc[v]);
        }
        __syncthreads();
    }
    for (int v = t; v < d.n; v += nt)
        d.len[v] = v == root ? 0.0 : d.rate[v] * (d.h[d.parent[v]] - d.h[v]);
    if (!d.grad) return;
    // height derivatives, then totals bottom-up
    for (int v = N + t; v < d.n; v += nt) {
        const int a = d.child[2 * (v - N)], b = d.child[2 * (v - N) + 1];
        d.G[v] = d.rate[a] * d.g[a] + d.rate[b] * d.g[b] - (v == root ? 0.0 : d.rate[v] * d.g[v]);
    }
    __syncthreads();
    for (int L = d.n_levels - 1; L >= 0; --L) {
        for (int k = d.level[L] + t; k < d.level[L + 1]; k += nt) {
            const int v = d.order[k];
            if (v < N) continue;
            double s = d.G[v];
            for (int c = 0; c < 2; ++c) {
                const int x = d.child[2 * (v - N) + c];
                if (x >= N) s += d.ratio[x - N] * d.G[x];
            }
            d.G[v] = s;
        }
        __syncthreads();
    }
    for (int v = N + t; v < d.n; v += nt)
        d.g_ratio[v - N] = v == root ? 0.0 : (d.h[d.parent[v]] - d.anc[v]) * d.G[v];
    for (int v = t; v < d.n; v += nt)
        d.g_rate[v] = v == root ? 0.0 : (d.h[d.parent[v]] - d.h[v]) * d.g[v];
    if (t == 0) d.g_root[0] = d.G[root];
}

// Host side: validate, order by depth, stage, launch, copy back.
int ratio_run(int n_tips, const int* parent, const double* tip_h, const double* ratio,
              double root_h, const double* rate, const double* grad, double* out_h,
              double* out_len, double* out_gr, double* out_groot, double* out_grate,
              void* stream, std::string* err) {
    auto bad = [&](const char* m) {
        *err = m;
        return TL_ERR_ARG;
    };
    if (n_tips < 2 || !parent || !tip_h || !ratio || !rate) return bad("null or short input");
    const int N = n_tips, n = 2 * N - 1, root = n - 1;
    std::vector<int> child(2 * (N - 1), -1), depth(n, 0);
    if (parent[root] != -1) return bad("the last node must be the root (parent -1)");
    for (int v = 0; v < root; ++v) {
        const int p = parent[v];
        if (p <= v || p < N || p >= n) return bad("parent[v] must be an internal node after v");
        int* c = &child[2 * (p - N)];
        if (c[0] < 0) c[0] = v;
        else if (c[1] < 0) c[1] = v;
        else return bad("a node has more than two children");
    }
    for (int k = 0; k < N - 1; ++k)
        if (child[2 * k + 1] < 0) return bad("an internal node has fewer than two children");
    for (int v = 0; v < n; ++v)
        if (!std::isfinite(rate[v]) || (v < N && !std::isfinite(tip_h[v])))
            return bad("non-finite rate or tip height");
    for (int k = 0; k < N - 2; ++k)
        if (!(ratio[k] > 0.0 && ratio[k] < 1.0)) return bad("ratios must lie in (0, 1)");
    for (int v = root - 1; v >= 0; --v) depth[v] = depth[parent[v]] + 1;
    const int n_levels = *std::max_element(depth.begin(), depth.end()) + 1;
    std::vector<int> level(n_levels + 1, 0), order(n);
    for (int v = 0; v < n; ++v) level[depth[v] + 1]++;
    for (int L = 0; L < n_levels; ++L) level[L + 1] += level[L];
    {
        std::vector<int> fill(level.begin(), level.end() - 1);
        for (int v = n - 1; v >= 0; --v) order[fill[depth[v]]++] = v;
    }
    // anchor below the root height
    {
        std::vector<double> anc(n);
        for (int v = 0; v < N; ++v) anc[v] = tip_h[v];
        for (int v = N; v < n; ++v) anc[v] = std::max(anc[child[2 * (v - N)]], anc[child[2 * (v - N) + 1]]);
        if (!(root_h > anc[root]) || !std::isfinite(root_h))
            return bad("the root height must exceed every tip height");
    }
    // one device block: ints then doubles
    const size_t ni = (size_t)n + 2 * (N - 1) + n + (n_levels + 1);
    const size_t nd = (size_t)N + (N - 1) + n + n + 4 * (size_t)n + (N - 1) + n + 1;
    std::vector<char> h(ni * sizeof(int) + 8 + nd * sizeof(double), 0);
    int* hi = reinterpret_cast<int*>(h.data());
    std::memcpy(hi, parent, sizeof(int) * n);
    std::memcpy(hi + n, child.data(), sizeof(int) * 2 * (N - 1));
    std::memcpy(hi + n + 2 * (N - 1), order.data(), sizeof(int) * n);
    std::memcpy(hi + 2 * n + 2 * (N - 1), level.data(), sizeof(int) * (n_levels + 1));
    const size_t dbl_off = ((ni * sizeof(int) + 7) / 8) * 8;
    double* hd = reinterpret_cast<double*>(h.data() + dbl_off);
    std::memcpy(hd, tip_h, sizeof(double) * N);
    std::memcpy(hd + N, ratio, sizeof(double) * (N - 1));
    std::memcpy(hd + 2 * N - 1, rate, sizeof(double) * n);
    if (grad) std::memcpy(hd + 2 * N - 1 + n, grad, sizeof(double) * n);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* d = nullptr;
    const size_t bytes = dbl_off + nd * sizeof(double);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), bytes, s);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return TL_ERR_OOM;
    }
    e = cudaMemcpyAsync(d, h.data(), bytes, cudaMemcpyHostToDevice, s);
    const int* di = reinterpret_cast<const int*>(d);
    double* dd = reinterpret_cast<double*>(d + dbl_off);
    RatioDev a;
    a.parent = di;
    a.child = di + n;
    a.order = di + n + 2 * (N - 1);
    a.level = di + 2 * n + 2 * (N - 1);
    a.tip_h = dd;
    a.ratio = dd + N;
    a.rate = dd + 2 * N - 1;
    a.g = dd + 2 * N - 1 + n;
    a.anc = dd + 2 * N - 1 + 2 * n;
    a.h = a.anc + n;
    a.len = a.h + n;
    a.G = a.len + n;
    a.g_ratio = a.G + n;
    a.g_rate = a.g_ratio + (N - 1);
    a.g_root = a.g_rate + n;
    a.root_h = root_h;
    a.n_tips = N;
    a.n = n;
    a.n_levels = n_levels;
    a.grad = grad != nullptr;
    if (e == cudaSuccess) {
        k_ratio<<<1, 1024, 0, s>>>(a);
        e = cudaGetLastError();
    }
    // results: [h | len] and [G | g_ratio | g_rate | g_root] are contiguous
    std::vector<double> out(2 * (size_t)n + n + (N - 1) + n + 1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.data(), a.h, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *err = cudaGetErrorString(e);
        return TL_ERR_CUDA;
    }
    const double* oh = out.data();
    const double* ol = oh + n;
    const double* ogr = oh + 3 * n;
    const double* ograte = ogr + (N - 1);
    if (out_h) std::memcpy(out_h, oh, sizeof(double) * n);
    if (out_len) std::memcpy(out_len, ol, sizeof(double) * n);
    if (out_gr) std::memcpy(out_gr, ogr, sizeof(double) * (N - 1));
    if (out_grate) std::memcpy(out_grate, ograte, sizeof(double) * n);
    if (out_groot) *out_groot = ograte[n];
    return TL_OK;
}

}  // namespace tl
