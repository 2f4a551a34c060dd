// api.cu -- host implementation of the C ABI declared in include/sclbm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace sclbm;

namespace {

thread_local char g_cuda_err[256] = "";

lb_status cuda_fail(cudaError_t e, const char *where) {
    std::snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", where, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return LB_ENOMEM;
    if (e == cudaErrorNotSupported) return LB_EUNSUPPORTED;
    return LB_ECUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// ---- stencil expansion (canonical pair order, see sclbm.h) ----------------
struct Group {
    std::array<int, 3> cb;  // sorted absolute components, descending
    double w;
};

bool lex_greater(const std::array<int, 3> &a, const std::array<int, 3> &b) {
    for (int k = 0; k < 3; ++k)
        if (a[k] != b[k]) return a[k] > b[k];
    return false;
}

// orbit of a base under permutations and sign flips (dim components)
std::vector<std::array<int, 3>> orbit(const std::array<int, 3> &cb, int dim) {
    std::vector<std::array<int, 3>> out;
    int perm[3] = {0, 1, 2};
    std::vector<int> idx(perm, perm + dim);
    std::sort(idx.begin(), idx.end());
    do {
        for (int s = 0; s < (1 << dim); ++s) {
            std::array<int, 3> v = {0, 0, 0};
            for (int k = 0; k < dim; ++k) {
                int c = cb[idx[k]];
                v[k] = (s >> k & 1) ? -c : c;
            }
            if (v[0] == 0 && v[1] == 0 && v[2] == 0) continue;
            if (std::find(out.begin(), out.end(), v) == out.end()) out.push_back(v);
        }
    } while (std::next_permutation(idx.begin(), idx.end()));
    return out;
}

bool is_rep(const std::array<int, 3> &v) {
    for (int k = 0; k < 3; ++k)
        if (v[k]) return v[k] > 0;
    return false;
}

double dfact(int k) {
    double r = 1;
    while (k > 1) { r *= k; k -= 2; }
    return r;
}

// Delta^{idx}: number of pairings of equal indices (zero if a count is odd).
double iso_tensor(const int *cnt) {
    double v = 1;
    for (int k = 0; k < 3; ++k) {
        if (cnt[k] % 2) return 0;
        v *= dfact(cnt[k] - 1);
    }
    return v;
}

lb_status expand(int dim, int n_groups, const int *base, const double *W,
                 std::vector<std::array<int, 3>> &vec, std::vector<double> &w,
                 std::vector<std::array<int, 3>> &gbase, std::vector<double> &gw,
                 lb_stencil_info *info) {
    if ((dim != 2 && dim != 3) || n_groups < 1 || !base || !W) return LB_EINVAL;
    std::vector<Group> gs;
    for (int g = 0; g < n_groups; ++g) {
        std::array<int, 3> a = {0, 0, 0};
        for (int k = 0; k < dim; ++k) {
            int c = base[g * dim + k];
            if (c < -LB_MAX_RADIUS || c > LB_MAX_RADIUS) return LB_EINVAL;
            a[k] = c < 0 ? -c : c;
        }
        std::sort(a.begin(), a.end(), [](int p, int q) { return p > q; });
        if (a[0] == 0) return LB_EINVAL;
        if (!std::isfinite(W[g])) return LB_EINVAL;
        for (auto &o : gs)
            if (o.cb == a) return LB_EINVAL;
        gs.push_back({a, W[g]});
    }
    std::stable_sort(gs.begin(), gs.end(), [](const Group &p, const Group &q) {
        int sp = p.cb[0] * p.cb[0] + p.cb[1] * p.cb[1] + p.cb[2] * p.cb[2];
        int sq = q.cb[0] * q.cb[0] + q.cb[1] * q.cb[1] + q.cb[2] * q.cb[2];
        if (sp != sq) return sp < sq;
        return lex_greater(p.cb, q.cb);
    });
    vec.clear();
    w.clear();
    gbase.clear();
    gw.clear();
    int radius = 0;
    for (auto &g : gs) {
        auto orb = orbit(g.cb, dim);
        std::vector<std::array<int, 3>> reps;
        for (auto &v : orb)
            if (is_rep(v)) reps.push_back(v);
        std::sort(reps.begin(), reps.end(), lex_greater);
        for (auto &v : reps) {
            vec.push_back(v);
            w.push_back(g.w);
        }
        gbase.push_back(g.cb);
        gw.push_back(g.w);
        radius = std::max(radius, g.cb[0]);
    }
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->n_groups = n_groups;
        info->n_pairs = (int)vec.size();
        info->n_vectors = 2 * (int)vec.size();
        info->radius = radius;
        auto mom = [&](int px, int py, int pz) {
            double s = 0;
            for (size_t a = 0; a < vec.size(); ++a) {
                double t = 2.0 * w[a];  // e and -e (even powers)
                for (int k = 0; k < px; ++k) t *= vec[a][0];
                for (int k = 0; k < py; ++k) t *= vec[a][1];
                for (int k = 0; k < pz; ++k) t *= vec[a][2];
                s += t;
            }
            return s;
        };
        info->e2 = mom(2, 0, 0);
        info->e4 = mom(2, 2, 0);
        info->e6 = mom(4, 2, 0) / 3.0;
        info->e8 = mom(4, 4, 0) / 9.0;
        for (int oi = 0; oi < 4; ++oi) {
            const int order = 4 + 2 * oi;
            // balanced reference tuple x^{2a} y^{2b}
            int a2 = ((order / 2 + 1) / 2) * 2, b2 = order - a2;
            int rc[3] = {a2, b2, 0};
            const double eref = mom(a2, b2, 0) / iso_tensor(rc);
            double worst = 0;
            for (int px = order; px >= 0; --px)
                for (int py = order - px; py >= 0; --py) {
                    int pz = order - px - py;
                    if (dim == 2 && pz) continue;
                    int cnt[3] = {px, py, pz};
                    double m = mom(px, py, pz);
                    double d = iso_tensor(cnt);
                    worst = std::max(worst, std::fabs(m - eref * d));
                }
            info->iso_residual[oi] = worst;
        }
    }
    return LB_OK;
}

// the D2Q9 / D3Q19 velocity tables in the state layout's order (host copies)
int vel9(int i, int k) {
    static const int t[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                                {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
    return t[i][k];
}
int vel19(int i, int k) {
    static const int t[19][3] = {
        {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1}, {-1, 0, -1},
        {1, 0, -1}, {-1, 0, 1}, {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[i][k];
}

void set_consts(lb_ctx *c) {
    double w[19];
    if (c->Q == 9) {
        w[0] = 4.0 / 9.0;
        for (int i = 1; i <= 4; ++i) w[i] = 1.0 / 9.0;
        for (int i = 5; i <= 8; ++i) w[i] = 1.0 / 36.0;
    } else {
        w[0] = 1.0 / 3.0;
        for (int i = 1; i <= 6; ++i) w[i] = 1.0 / 18.0;
        for (int i = 7; i <= 18; ++i) w[i] = 1.0 / 36.0;
    }
    const double tau = c->p.tau;
    c->k.omega = 1.0 / tau;
    const double pref = 1.0 - 1.0 / (2.0 * tau);
    for (int i = 0; i < 19; ++i) {
        c->k.w[i] = i < c->Q ? w[i] : 0.0;
        c->k.cw[i] = i < c->Q ? pref * w[i] : 0.0;
    }
    c->Gp = c->p.g_convention == LB_G_TIMES_CS2 ? c->p.G / 3.0 : c->p.G;
    c->k.mGp = -c->Gp;
    c->k.rho0 = c->p.rho0_shift;
    c->k.kA = c->p.forcing_A / tau;
    c->k.psi_kind = c->p.psi_kind;
    c->k.psi_eps = c->p.psi_kind == LB_PSI_EPS ? c->p.psi_eps : 0.0;
    c->k.psi_inv = c->p.psi_kind == LB_PSI_EPS ? 1.0 / c->p.psi_eps : 0.0;
    fill_mass_exact_f32(c->k, c->Q);
}

size_t tsize(const lb_ctx *c) { return c->p.precision == LB_FP64 ? 8 : 4; }

// populations of one state chunk that fit the staging buffer as binary64
int stage_pops(lb_ctx *c) {
    const long long per = (long long)(stage_bytes(c) / (sizeof(double) * (size_t)c->g.N));
    return (int)(per < c->Q ? per : c->Q);
}

lb_status check_flags(lb_ctx *c, Flags *h) {
    CK(cudaMemcpyAsync(h, c->flags, sizeof(Flags), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h->timeouts) {
        std::snprintf(g_cuda_err, sizeof g_cuda_err,
                      "fused kernel: %llu bounded barrier waits gave up", h->timeouts);
        return LB_ECUDA;
    }
    return h->err_step != ULLONG_MAX ? LB_EUNSTABLE : LB_OK;
}

}  // namespace

void lb_set_error_message(const char *msg) {
    std::snprintf(g_cuda_err, sizeof g_cuda_err, "%s", msg);
}

namespace sclbm {

void tm_begin(lb_ctx *c, int kind) {
    if (!c->timing) return;
    if (c->ev_used + 2 > c->ev_cap) {
        int cap = c->ev_cap ? 2 * c->ev_cap : 256;
        cudaEvent_t *ev = (cudaEvent_t *)std::realloc(c->ev, cap * sizeof(cudaEvent_t));
        int *kd = (int *)std::realloc(c->ev_kind, (cap / 2) * sizeof(int));
        if (!ev || !kd) {  // out of host memory: stop timing, keep stepping
            if (ev) c->ev = ev;
            if (kd) c->ev_kind = kd;
            c->timing = false;
            return;
        }
        c->ev = ev;
        c->ev_kind = kd;
        for (int i = c->ev_cap; i < cap; ++i) cudaEventCreate(&c->ev[i]);
        c->ev_cap = cap;
    }
    c->ev_kind[c->ev_used / 2] = kind;
    cudaEventRecord(c->ev[c->ev_used], c->stream);
}

void tm_end(lb_ctx *c) {
    if (!c->timing) return;
    cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
    c->ev_used += 2;
}

}  // namespace sclbm

extern "C" {

lb_status lb_timing(lb_ctx *c, int enable) {
    if (!c) return LB_EINVAL;
    if (enable) {
        CK(cudaStreamSynchronize(c->stream));
        c->ev_used = 0;
        for (int k = 0; k < LB_KERNEL_KINDS; ++k) {
            c->kind_ms[k] = 0.0;
            c->kind_n[k] = 0;
        }
    }
    c->timing = enable != 0;
    return LB_OK;
}

lb_status lb_timing_read(lb_ctx *c, double *ms, long long *launches) {
    if (!c) return LB_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    for (int e = 0; e < c->ev_used; e += 2) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->ev[e], c->ev[e + 1]));
        c->kind_ms[c->ev_kind[e / 2]] += t;
        c->kind_n[c->ev_kind[e / 2]] += 1;
    }
    c->ev_used = 0;
    for (int k = 0; k < LB_KERNEL_KINDS; ++k) {
        if (ms) ms[k] = c->kind_ms[k];
        if (launches) launches[k] = c->kind_n[k];
    }
    return LB_OK;
}


const char *lb_status_str(lb_status s) {
    switch (s) {
        case LB_OK: return "LB_OK";
        case LB_EINVAL: return "LB_EINVAL: invalid argument";
        case LB_ENOMEM: return "LB_ENOMEM: out of memory";
        case LB_ECUDA: return "LB_ECUDA: CUDA runtime error";
        case LB_EUNSTABLE: return "LB_EUNSTABLE: density check failed (n <= 0 or NaN)";
        case LB_EUNSUPPORTED: return "LB_EUNSUPPORTED: not covered by the library";
        case LB_ESTATE: return "LB_ESTATE: call out of order";
    }
    return "unknown lb_status";
}

const char *lb_last_cuda_error(void) { return g_cuda_err; }

lb_status lb_params_default(lb_params *p) {
    if (!p) return LB_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->lattice = LB_D2Q9;
    p->nx = 64;
    p->ny = 64;
    p->nz = 1;
    p->precision = LB_FP64;
    p->tau = 1.0;
    p->G = -5.0;
    p->g_convention = LB_G_LITERAL;
    p->psi_kind = LB_PSI_EXP;
    p->psi_eps = 0.0;
    p->rho0_shift = 0.5;
    p->forcing_A = 0.0;
    return LB_OK;
}

lb_status lb_expand_stencil(int dim, int n_groups, const int *base_vectors, const double *W,
                            int max_pairs, int *pair_vec, double *pair_w, int *n_pairs,
                            lb_stencil_info *info) {
    std::vector<std::array<int, 3>> vec, gb;
    std::vector<double> w, gw;
    lb_status s = expand(dim, n_groups, base_vectors, W, vec, w, gb, gw, info);
    if (s != LB_OK) return s;
    if ((int)vec.size() > max_pairs && (pair_vec || pair_w)) return LB_EINVAL;
    if (n_pairs) *n_pairs = (int)vec.size();
    for (size_t a = 0; a < vec.size() && (int)a < max_pairs; ++a) {
        if (pair_vec)
            for (int k = 0; k < 3; ++k) pair_vec[3 * a + k] = vec[a][k];
        if (pair_w) pair_w[a] = w[a];
    }
    return LB_OK;
}

// flag = 1 if any rho[s], s < N, is not positive and finite
__global__ void k_check_rho(const double *__restrict__ rho, long long N, unsigned int *flag) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += stride) {
        const double r = rho[s];
        if (!(r > 0.0 && r <= 1.7976931348623157e308)) *flag = 1u;
    }
}

lb_status lb_create(const lb_params *p, const double *rho_init, const double *u_init,
                    void *cuda_stream, lb_ctx **out) {
    if (!p || !rho_init || !out) return LB_EINVAL;
    *out = nullptr;
    if (p->lattice != LB_D2Q9 && p->lattice != LB_D3Q19) return LB_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LB_EINVAL;
    if (p->lattice == LB_D2Q9 && p->nz != 1) return LB_EINVAL;
    if (p->precision != LB_FP64 && p->precision != LB_FP32_SHIFTED) return LB_EINVAL;
    if (!(p->tau > 0.5) || !std::isfinite(p->tau) || !std::isfinite(p->G)) return LB_EINVAL;
    if (p->g_convention != LB_G_LITERAL && p->g_convention != LB_G_TIMES_CS2) return LB_EINVAL;
    if (p->psi_kind != LB_PSI_EXP && p->psi_kind != LB_PSI_EPS) return LB_EINVAL;
    if (p->psi_kind == LB_PSI_EPS && !(p->psi_eps > 0.0 && std::isfinite(p->psi_eps)))
        return LB_EINVAL;
    if (!std::isfinite(p->rho0_shift) || !std::isfinite(p->forcing_A)) return LB_EINVAL;
    const long long N = (long long)p->nx * p->ny * p->nz;

    lb_ctx *c = new (std::nothrow) lb_ctx();
    if (!c) return LB_ENOMEM;
    c->p = *p;
    c->D = p->lattice == LB_D2Q9 ? 2 : 3;
    c->Q = p->lattice == LB_D2Q9 ? 9 : 19;
    // shifted-FP32 D3Q19 lattices that tile exactly get periodic ghost
    // columns and rows (3 each side) for the TMA kernel.  Node (0, 0) sits 32
    // columns into a padded row (rows are nx + 64 floats, a multiple of 128
    // bytes): every warp's row of 32 nodes is one whole 128-byte line, so a
    // step's stores never write part of a line or sector (measured at 256^3:
    // 0.592 ms per step with the interior 4 columns in, 0.567 at 8, 0.555 at
    // 16, 0.540 at 32); the 8 columns next to each edge are kept as images
    c->padded = p->precision == LB_FP32_SHIFTED && p->lattice == LB_D3Q19 && p->nx % 32 == 0 &&
                p->ny % 8 == 0 && p->nz >= 8;
    const int ox = c->padded ? 32 : 0, oy = c->padded ? 3 : 0;
    c->g = {p->nx, p->ny, p->nz, N, p->nx + 2 * ox, p->ny + 2 * oy, ox, oy,
            (long long)(p->nx + 2 * ox) * (p->ny + 2 * oy) * p->nz};
    set_consts(c);
    c->cur = 0;
    c->fused_enabled = true;
    c->fused_tma = true;
    c->wait_polls = 1LL << 26;
    c->fused_zchunk = 28;
    auto fail = [&](lb_status s) {
        lb_destroy(c);
        return s;
    };
    cudaError_t e;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
        c->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreate"));
        c->own_stream = true;
    }
    const size_t fbytes = (size_t)c->Q * c->g.Np * tsize(c);
    for (int b = 0; b < 2; ++b) {
        e = cudaMalloc(&c->f[b], fbytes);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(f)"));
    }
    // binary32 lattices below 2^31 nodes keep psi with a periodic halo of
    // PSI_HALO nodes (the generic kernels' branch-free stencil offsets)
    {
        const long long H = PSI_HALO, Hz = c->D == 3 ? H : 0;
        const long long halo_n = (p->nx + 2 * H) * (p->ny + 2 * H) * (p->nz + 2 * Hz);
        c->psi_halo = (p->precision == LB_FP32_SHIFTED && halo_n < (1LL << 31)) ? PSI_HALO : 0;
        const size_t np = c->psi_halo ? (size_t)halo_n : (size_t)N;
        e = cudaMalloc(&c->psi, np * tsize(c));
    }
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(psi)"));
    e = cudaMalloc(&c->flags, sizeof(Flags));
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(flags)"));
    e = cudaMalloc(&c->red, 1024 * 128);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(red)"));
    Flags h0 = {ULLONG_MAX, 0, 0, 0, 0};
    e = cudaMemcpyAsync(c->flags, &h0, sizeof h0, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy(flags)"));
    if (c->padded) {
        e = cudaMemsetAsync(c->f[0], 0, fbytes, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->f[1], 0, fbytes, c->stream);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemset(f)"));
        c->tma_ok = tma_make_maps(c);
    }
    // the initial density (and velocity) are staged in the second population
    // buffer, which the first step overwrites: no scratch allocation
    if ((size_t)(1 + c->D) * N * sizeof(double) > stage_bytes(c)) return fail(LB_EINVAL);
    double *rho_d = stage_ptr(c), *u_d = u_init ? rho_d + N : nullptr;
    e = cudaMemcpyAsync(rho_d, rho_init, N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy(rho)"));
    if (u_init) {
        e = cudaMemcpyAsync(u_d, u_init, c->D * N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy(u)"));
    }
    // every initial density positive and finite: checked on the device after
    // the upload (a host loop over the N values took about 10 ms at 256^3),
    // the flag in the reduction buffer's first word
    unsigned int *bad_d = reinterpret_cast<unsigned int *>(c->red);
    e = cudaMemsetAsync(bad_d, 0, sizeof(unsigned int), c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemset(flag)"));
    const int gb = (int)std::max(1LL, std::min((N + 255) / 256, 152LL * 32));
    k_check_rho<<<gb, 256, 0, c->stream>>>(rho_d, N, bad_d);
    e = p->precision == LB_FP64 ? f64_init(c, rho_d, u_d) : f32_init(c, rho_d, u_d);
    if (e != cudaSuccess) return fail(cuda_fail(e, "init kernel"));
    unsigned int bad = 0;
    e = cudaMemcpyAsync(&bad, bad_d, sizeof bad, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy(flag)"));
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(cuda_fail(e, "lb_create sync"));
    if (bad) return fail(LB_EINVAL);
    *out = c;
    return LB_OK;
}

lb_status lb_destroy(lb_ctx *c) {
    if (!c) return LB_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph_valid) cudaGraphExecDestroy(c->graph);
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->psi);
    cudaFree(c->red);
    cudaFree(c->flags);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    for (int i = 0; i < c->ev_cap; ++i) cudaEventDestroy(c->ev[i]);
    std::free(c->ev);
    std::free(c->ev_kind);
    delete c;
    return LB_OK;
}

namespace {

// steps per replay of a context's CUDA graph (even: the buffer parity
// returns to where it started)
constexpr int kStepGraph = 32;

cudaError_t one_step(lb_ctx *c) { return c->p.precision == LB_FP64 ? f64_step(c) : f32_step(c); }

void drop_graph(lb_ctx *c) {
    if (c->graph_valid) cudaGraphExecDestroy(c->graph);
    c->graph_valid = false;
}

// Capture kStepGraph steps of the context's stream into c->graph (nothing
// runs during the capture; the host-side buffer parity and launch count are
// restored).
lb_status build_step_graph(lb_ctx *c) {
    drop_graph(c);
    const int cur0 = c->cur;
    const long long l0 = c->launches;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "step graph capture");
    for (int t = 0; t < kStepGraph && e == cudaSuccess; ++t) e = one_step(c);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    c->graph_launches = c->launches - l0;
    c->launches = l0;
    c->cur = cur0;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "step graph");
    c->graph_valid = true;
    c->graph_cur = cur0;
    return LB_OK;
}

}  // namespace

lb_status lb_set_stencil(lb_ctx *c, int n_groups, const int *base_vectors, const double *W,
                         lb_stencil_info *info) {
    if (!c) return LB_EINVAL;
    std::vector<std::array<int, 3>> vec, gb;
    std::vector<double> w, gw;
    lb_stencil_info tmp;
    lb_status s = expand(c->D, n_groups, base_vectors, W, vec, w, gb, gw, &tmp);
    if (s != LB_OK) return s;
    if ((int)vec.size() > MAXP) return LB_EINVAL;
    c->pairs64.npairs = c->pairs32.npairs = (int)vec.size();
    c->pairs64.radius = c->pairs32.radius = tmp.radius;
    for (size_t a = 0; a < vec.size(); ++a) {
        for (int k = 0; k < 3; ++k) {
            c->pairs64.v[a][k] = (signed char)vec[a][k];
            c->pairs32.v[a][k] = (signed char)vec[a][k];
        }
        c->pairs64.w[a] = w[a];
        c->pairs32.w[a] = (float)w[a];
    }
    // the binary32 generic kernels' interior form of the stencil
    {
        PairsFast &F = c->pfast;
        std::memset(&F, 0, sizeof F);
        F.npairs = (int)vec.size();
        F.R = std::max(1, tmp.radius);
        F.H = c->psi_halo;
        F.Hz = c->D == 3 ? c->psi_halo : 0;
        F.pxp = c->g.nx + 2 * F.H;
        F.pyp = c->g.ny + 2 * F.H;
        F.pull_pad = c->g.ox > 0 && c->g.oy > 0;
        for (size_t a = 0; a < vec.size(); ++a) {
            F.nb[a] = (vec[a][2] * F.pyp + vec[a][1]) * F.pxp + vec[a][0];
            F.nbs[a] = (vec[a][2] * ct_by(c->D) + vec[a][1]) * CT_BX + vec[a][0];
            for (int k = 0; k < 3; ++k) F.we[a][k] = (float)(w[a] * (double)vec[a][k]);
        }
        for (int i = 0; i < c->Q; ++i) {
            int cv[3];
            for (int k = 0; k < 3; ++k) cv[k] = c->Q == 9 ? vel9(i, k) : vel19(i, k);
            F.pop[i] = (cv[2] * c->g.nyp + cv[1]) * c->g.nxp + cv[0];
        }
    }
    c->n_groups = (int)gb.size();
    c->e2 = tmp.e2;
    for (size_t g = 0; g < gb.size(); ++g) {
        for (int k = 0; k < 3; ++k) c->group_base[g][k] = gb[g][k];
        c->group_w[g] = gw[g];
    }
    c->stencil_set = true;
    c->fast3d_ok = fused3d_applicable(c, c->fused_W, &c->fused_ng);
    c->fast2d_ok = fused2d_applicable(c, c->fused2d_W);
    drop_graph(c);
    if (info) *info = tmp;
    return LB_OK;
}

lb_status lb_step(lb_ctx *c, int nsteps) {
    if (!c || nsteps < 0) return LB_EINVAL;
    if (!c->stencil_set) return LB_ESTATE;
    int t = 0;
    // long runs replay a captured graph of kStepGraph steps (not while
    // per-kernel timing records events); the steps before the first replay
    // run directly, so every kernel has been launched once before a capture
    if (nsteps >= 3 * kStepGraph && !c->timing) {
        for (; t < 2; ++t) {
            cudaError_t e = one_step(c);
            if (e != cudaSuccess) return cuda_fail(e, "step kernels");
        }
        if (c->graph_valid && c->graph_cur != c->cur) {
            cudaError_t e = one_step(c);
            if (e != cudaSuccess) return cuda_fail(e, "step kernels");
            ++t;
        }
        if (!c->graph_valid) {
            lb_status s = build_step_graph(c);
            if (s != LB_OK) return s;
        }
        for (; nsteps - t >= kStepGraph; t += kStepGraph) {
            cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "step graph launch");
            c->launches += c->graph_launches;
        }
    }
    for (; t < nsteps; ++t) {
        cudaError_t e = one_step(c);
        if (e != cudaSuccess) return cuda_fail(e, "step kernels");
    }
    c->steps += nsteps;
    return LB_OK;
}

lb_status lb_sync(lb_ctx *c) {
    if (!c) return LB_EINVAL;
    Flags h;
    return check_flags(c, &h);
}

lb_status lb_observables(lb_ctx *c, lb_obs *out) {
    if (!c || !out) return LB_EINVAL;
    if (!c->stencil_set) return LB_ESTATE;
    cudaError_t e = obs_fused(c);
    if (e != cudaSuccess) return cuda_fail(e, "observables kernels");
    double h[7];
    CK(cudaMemcpyAsync(h, obs_results(c), sizeof h, cudaMemcpyDeviceToHost, c->stream));
    Flags f;
    lb_status st = check_flags(c, &f);
    if (st != LB_OK && st != LB_EUNSTABLE) return st;
    out->mass = h[0];
    for (int k = 0; k < 3; ++k) out->mom[k] = k < c->D ? h[1 + k] : 0.0;
    out->umax = h[4];
    out->rho_min = h[5];
    out->rho_max = h[6];
    out->step = c->steps;
    out->error_step = f.err_step == ULLONG_MAX ? -1 : (long long)f.err_step;
    out->exp_ambiguous = (long long)f.exp_amb;
    return st;
}

lb_status lb_pressure_tensor(lb_ctx *c, double *out) {
    if (!c || !out) return LB_EINVAL;
    if (!c->stencil_set) return LB_ESTATE;
    const long long N = c->g.N;
    const int nc = c->D == 2 ? 3 : 6;
    if ((size_t)(1 + nc) * N * sizeof(double) > stage_bytes(c)) return LB_EUNSUPPORTED;
    double *psi = stage_ptr(c), *P = psi + N;
    cudaError_t e = ptensor_field(c, psi, P);
    if (e == cudaErrorNotSupported) return LB_EUNSUPPORTED;
    if (e != cudaSuccess) return cuda_fail(e, "pressure tensor kernels");
    CK(cudaMemcpyAsync(out, P, (size_t)nc * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_flat_interfaces(lb_ctx *c, int max_interfaces, lb_flat_obs *out, int *n_found) {
    if (!c || max_interfaces < 0 || (max_interfaces > 0 && !out)) return LB_EINVAL;
    if (!c->stencil_set) return LB_ESTATE;
    const int maxw = max_interfaces < 256 ? max_interfaces : 256;
    int *cnt = reinterpret_cast<int *>(obs_results(c) + 8);
    lb_flat_obs *res = reinterpret_cast<lb_flat_obs *>(obs_results(c) + 16);
    cudaError_t e = flat_interfaces(c, maxw, res, cnt);
    if (e == cudaErrorNotSupported) return LB_EUNSUPPORTED;
    if (e == cudaErrorInvalidValue) return LB_EINVAL;
    if (e != cudaSuccess) return cuda_fail(e, "flat interface kernels");
    int k = 0;
    CK(cudaMemcpyAsync(&k, cnt, sizeof k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int m = k < maxw ? k : maxw;
    if (m > 0)
        CK(cudaMemcpyAsync(out, res, (size_t)m * sizeof(lb_flat_obs), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (n_found) *n_found = k;
    return LB_OK;
}

lb_status lb_curved_interface(lb_ctx *c, const double *center, lb_curved_obs *out) {
    if (!c || !center || !out) return LB_EINVAL;
    if (!c->stencil_set) return LB_ESTATE;
    const int ext[3] = {c->g.nx, c->g.ny, c->g.nz};
    for (int k = 0; k < c->D; ++k)
        if (!(center[k] >= 0.0 && center[k] < ext[k])) return LB_EINVAL;
    lb_curved_obs *res = reinterpret_cast<lb_curved_obs *>(obs_results(c) + 16);
    double cen[3] = {center[0], center[1], c->D == 3 ? center[2] : 0.0};
    cudaError_t e = curved_interface(c, cen, c->e2, res);
    if (e == cudaErrorNotSupported) return LB_EUNSUPPORTED;
    if (e == cudaErrorInvalidValue) return LB_EINVAL;
    if (e != cudaSuccess) return cuda_fail(e, "curved interface kernels");
    CK(cudaMemcpyAsync(out, res, sizeof *out, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!(out->n_in != out->n_out)) return LB_EINVAL;   // no interface
    return LB_OK;
}

namespace {
// least-squares line y = a x + b
bool fit_line(const double *x, const double *y, int n, double *a, double *b) {
    double sx = 0, sy = 0;
    for (int i = 0; i < n; ++i) { sx += x[i]; sy += y[i]; }
    const double mx = sx / n, my = sy / n;
    double sxx = 0, sxy = 0;
    for (int i = 0; i < n; ++i) {
        sxx += (x[i] - mx) * (x[i] - mx);
        sxy += (x[i] - mx) * (y[i] - my);
    }
    if (!(sxx > 0)) return false;
    *a = sxy / sxx;
    *b = my - *a * mx;
    return true;
}
}  // namespace

lb_status lb_fit_laplace(const lb_curved_obs *runs, int n, int dim, double *sigma,
                         double *intercept) {
    if (!runs || n < 2 || (dim != 2 && dim != 3) || !sigma) return LB_EINVAL;
    std::vector<double> x(n), y(n);
    for (int i = 0; i < n; ++i) {
        const double sg = runs[i].bubble ? -1.0 : 1.0;
        x[i] = sg / runs[i].R_e;
        y[i] = sg * runs[i].dP;
    }
    double a, b;
    if (!fit_line(x.data(), y.data(), n, &a, &b)) return LB_EINVAL;
    *sigma = a / (dim - 1);
    if (intercept) *intercept = b;
    return LB_OK;
}

lb_status lb_fit_tolman(const lb_curved_obs *runs, int n, int dim, double sigma0, double *delta,
                        double *intercept) {
    if (!runs || n < 2 || (dim != 2 && dim != 3) || !delta || !(sigma0 != 0.0)) return LB_EINVAL;
    std::vector<double> x(n), y(n);
    for (int i = 0; i < n; ++i) {
        const double sg = runs[i].bubble ? -1.0 : 1.0;
        x[i] = sg / runs[i].R_s;
        y[i] = runs[i].dP * runs[i].R_s / ((dim - 1) * sigma0);
    }
    double a, b;
    if (!fit_line(x.data(), y.data(), n, &a, &b)) return LB_EINVAL;
    *delta = -a / (dim - 1);
    if (intercept) *intercept = b;
    return LB_OK;
}

lb_status lb_get_fields(lb_ctx *c, double *rho, double *u) {
    if (!c) return LB_EINVAL;
    if (!c->stencil_set) return LB_ESTATE;
    const long long N = c->g.N;
    if ((size_t)(2 + c->D) * N * sizeof(double) > stage_bytes(c)) return LB_EUNSUPPORTED;
    double *n = stage_ptr(c), *ud = n + 2 * N;
    cudaError_t e;
    if (!u)   // the density alone: no psi, no force
        e = c->p.precision == LB_FP64 ? f64_density_psi(c, n, nullptr) : f32_density_psi(c, n, nullptr);
    else
        e = c->p.precision == LB_FP64 ? f64_fields(c, n, ud, nullptr) : f32_fields(c, n, ud, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "fields kernels");
    if (rho) CK(cudaMemcpyAsync(rho, n, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (u) CK(cudaMemcpyAsync(u, ud, c->D * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_get_state(lb_ctx *c, double *f) {
    if (!c || !f) return LB_EINVAL;
    const long long N = c->g.N;
    const int chunk = stage_pops(c);
    if (chunk < 1) return LB_EUNSUPPORTED;
    double *st = stage_ptr(c);
    for (int i0 = 0; i0 < c->Q; i0 += chunk) {
        const int i1 = i0 + chunk < c->Q ? i0 + chunk : c->Q;
        cudaError_t e = c->p.precision == LB_FP64 ? f64_get_state(c, st, i0, i1) : f32_get_state(c, st, i0, i1);
        if (e != cudaSuccess) return cuda_fail(e, "get_state kernel");
        CK(cudaMemcpyAsync(f + (size_t)i0 * N, st, (size_t)(i1 - i0) * N * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_set_state(lb_ctx *c, const double *f) {
    if (!c || !f) return LB_EINVAL;
    const long long N = c->g.N;
    const int chunk = stage_pops(c);
    if (chunk < 1) return LB_EUNSUPPORTED;
    double *st = stage_ptr(c);
    for (int i0 = 0; i0 < c->Q; i0 += chunk) {
        const int i1 = i0 + chunk < c->Q ? i0 + chunk : c->Q;
        CK(cudaMemcpyAsync(st, f + (size_t)i0 * N, (size_t)(i1 - i0) * N * sizeof(double),
                           cudaMemcpyHostToDevice, c->stream));
        cudaError_t e = c->p.precision == LB_FP64 ? f64_set_state(c, st, i0, i1) : f32_set_state(c, st, i0, i1);
        if (e != cudaSuccess) return cuda_fail(e, "set_state kernel");
    }
    if (c->p.precision != LB_FP64) {
        cudaError_t e = ghosts_refresh(c);
        if (e != cudaSuccess) return cuda_fail(e, "ghost refresh");
    }
    CK(cudaStreamSynchronize(c->stream));
    return LB_OK;
}

lb_status lb_exp_cr(const double *x, double *y, long long n, long long *n_ambiguous) {
    if (n < 0 || (n > 0 && (!x || !y))) return LB_EINVAL;
    if (n_ambiguous) *n_ambiguous = 0;
    if (n == 0) return LB_OK;
    double *d = nullptr;
    unsigned long long *amb = nullptr;
    CK(cudaMalloc(&d, 2 * n * sizeof(double) + 16));
    amb = (unsigned long long *)(d + 2 * n);
    cudaError_t e = cudaMemcpy(d, x, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(amb, 0, sizeof *amb);
    if (e == cudaSuccess) e = exp_batch(d, d + n, n, amb, 0);
    if (e == cudaSuccess) e = cudaMemcpy(y, d + n, n * sizeof(double), cudaMemcpyDeviceToHost);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, amb, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "lb_exp_cr");
    if (n_ambiguous) *n_ambiguous = (long long)h;
    return LB_OK;
}

lb_status lb_psi_eval(int psi_kind, double psi_eps, const double *n_in, double *psi, long long n,
                      long long *n_ambiguous) {
    if (psi_kind != LB_PSI_EXP && psi_kind != LB_PSI_EPS) return LB_EINVAL;
    if (psi_kind == LB_PSI_EPS && !(psi_eps > 0.0 && std::isfinite(psi_eps))) return LB_EINVAL;
    if (n < 0 || (n > 0 && (!n_in || !psi))) return LB_EINVAL;
    if (n_ambiguous) *n_ambiguous = 0;
    for (long long k = 0; k < n; ++k)
        if (!(n_in[k] > 0.0) || !std::isfinite(n_in[k])) return LB_EINVAL;
    if (n == 0) return LB_OK;
    double *d = nullptr;
    CK(cudaMalloc(&d, 2 * n * sizeof(double) + 16));
    unsigned long long *amb = (unsigned long long *)(d + 2 * n);
    cudaError_t e = cudaMemcpy(d, n_in, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(amb, 0, sizeof *amb);
    if (e == cudaSuccess) e = psi_batch(d, d + n, n, psi_kind, psi_eps, amb, 0);
    if (e == cudaSuccess) e = cudaMemcpy(psi, d + n, n * sizeof(double), cudaMemcpyDeviceToHost);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, amb, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "lb_psi_eval");
    if (n_ambiguous) *n_ambiguous = (long long)h;
    return LB_OK;
}

long long lb_kernel_launches(const lb_ctx *c) { return c ? c->launches : 0; }

lb_status lb_device_counters(lb_ctx *c, long long out[5]) {
    if (!c || !out) return LB_EINVAL;
    Flags h;
    CK(cudaMemcpyAsync(&h, c->flags, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out[0] = h.err_step == ULLONG_MAX ? -1 : (long long)h.err_step;
    out[1] = (long long)h.step;
    out[2] = (long long)h.exp_amb;
    out[3] = (long long)h.blocks_done;
    out[4] = (long long)h.timeouts;
    return LB_OK;
}

lb_status lb_set_option(lb_ctx *c, int option, long long value) {
    if (!c) return LB_EINVAL;
    drop_graph(c);   // the captured steps bake the options in
    switch (option) {
        case LB_OPT_FUSED:
            c->fused_enabled = value != 0;
            return LB_OK;
        case LB_OPT_TMA:
            c->fused_tma = value != 0;
            return LB_OK;
        case LB_OPT_ZCHUNK:
            if (value < 1 || value > 1 << 20) return LB_EINVAL;
            c->fused_zchunk = (int)value;
            return LB_OK;
        case LB_OPT_WAIT_POLLS:
            if (value < 0 || value > (1LL << 40)) return LB_EINVAL;
            c->wait_polls = value;
            return LB_OK;
    }
    return LB_EINVAL;
}

int lb_fused_active(const lb_ctx *c) {
    if (!(c && c->stencil_set && c->fused_enabled)) return 0;
    if (c->Q == 9) return c->fast2d_ok ? 3 : 0;
    if (!c->fast3d_ok) return 0;
    return c->tma_ok && c->fused_tma ? 2 : 1;
}

}  // extern "C"
