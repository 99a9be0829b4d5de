// C ABI of the cascading-smoother multigrid library (see
// include/cascade_mg.h): handle management, the V-cycle of Algorithm 1
// enqueued level by level and captured once into a CUDA graph, and the solve
// drivers (stationary iteration, FP64 iterative refinement around an FP32
// cycle, and left-preconditioned restarted GMRES as in Sec. 3.1).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <string>

#include "cs_internal.cuh"

namespace csx {

static thread_local std::string g_err;
static thread_local bool g_serial_levels = false;
std::atomic<int64_t> g_launches{0};

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

cs_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return e == cudaErrorMemoryAllocation ? CS_ERR_NOMEM : CS_ERR_CUDA;
}

static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {nullptr};

static cs_status pool_for_current_device(cudaMemPool_t *out) {
    int dev = 0;
    CSX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device ordinal %d unsupported", dev); return CS_ERR_UNSUPPORTED; }
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        CSX_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = ~(uint64_t)0;  // retain freed memory for the next setup
        CSX_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return CS_OK;
}

cs_status dalloc(void **p, size_t bytes, int64_t *acct, cudaStream_t s) {
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    CSX_TRY(pool_for_current_device(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return CS_ERR_NOMEM;
    }
    if (acct) *acct += (int64_t)bytes;
    return CS_OK;
}

void dfree(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

static bool is_star_offset(int dim, const int *o) {
    int nz = (o[0] != 0) + (o[1] != 0) + (o[2] != 0);
    if (dim == 2 && o[2] != 0) return false;
    return nz <= 1;
}
static int star_slot(const int *o) {
    if (o[0] == -1) return 1;
    if (o[0] == 1) return 2;
    if (o[1] == -1) return 3;
    if (o[1] == 1) return 4;
    if (o[2] == -1) return 5;
    if (o[2] == 1) return 6;
    return 0;
}
static int box_slot(int dim, const int *o) { return (o[0] + 1) + 3 * (o[1] + 1) + (dim == 3 ? 9 * (o[2] + 1) : 0); }

static void fill_offsets(Level &L) {
    for (int s = 0; s < L.nst; ++s) {
        int *o = L.off[s];
        o[0] = o[1] = o[2] = 0;
        if (L.kind == STAR) {
            if (s == 1) o[0] = -1;
            else if (s == 2) o[0] = 1;
            else if (s == 3) o[1] = -1;
            else if (s == 4) o[1] = 1;
            else if (s == 5) o[2] = -1;
            else if (s == 6) o[2] = 1;
        } else {
            o[0] = s % 3 - 1;
            o[1] = (s / 3) % 3 - 1;
            o[2] = L.g.dim == 3 ? s / 9 - 1 : 0;
        }
    }
}

// --------------------------------------------------------------- V-cycle
template <typename T>
struct View {
    const T *A;
    const T *lam;
    T *b, *x, *t;
};

template <typename T>
static View<T> view(const cs_hierarchy *h, const cs_cascade *c, int l);
template <>
View<double> view<double>(const cs_hierarchy *h, const cs_cascade *c, int l) {
    const Level &L = h->lev[l];
    return {L.A, l < c->nlev ? c->lam[l] : nullptr, L.b, L.x, L.t};
}
template <>
View<float> view<float>(const cs_hierarchy *, const cs_cascade *c, int l) {
    const LowLevel &L = c->lo[l];
    return {L.A, L.lam, L.b, L.x, L.t};
}
template <>
View<__nv_bfloat16> view<__nv_bfloat16>(const cs_hierarchy *, const cs_cascade *c, int l) {
    const LowLevel16 &L = c->lo16[l];
    return {L.A, L.lam, L.b, L.x, L.t};
}

// doubles of Lambda per cascade step on a level
static int64_t lam_step(const Level &L) { return L.bs > 1 ? L.nblocks * L.nmax * L.nmax : L.g.N; }

static void set_blocks(Level &L, int bs) {
    L.bs = bs;
    L.nbx = (L.g.nx + bs - 1) / bs;
    L.nby = (L.g.ny + bs - 1) / bs;
    L.nbz = L.g.dim == 3 ? (L.g.nz + bs - 1) / bs : 1;
    L.nblocks = (int64_t)L.nbx * L.nby * L.nbz;
    L.nmax = L.g.dim == 3 ? bs * bs * bs : bs * bs;
}

static bool inplace_colours(const cs_cascade *c, const Level &L) {
    // red-black is a graph colouring of a STAR stencil: colour-k updates read
    // only the other colour, so they may overwrite x in place
    return c->kind == CS_MULTIPLICATIVE && L.kind == STAR;
}

// one application of the cascade on level l; `cur` is the buffer holding the
// iterate (updated); `xzero` marks an all-zero iterate (cleared on return)
template <typename T>
static cs_status smooth_apply(const cs_hierarchy *h, const cs_cascade *c, int l, const View<T> &v, const T *b,
                              T *&cur, T *&other, bool reverse, bool &xzero, cudaStream_t s) {
    const Level &L = h->lev[l];
    const bool inpl = inplace_colours(c, L);
    for (int step = 0; step < c->nu; ++step) {
        int lv = reverse ? c->nu - 1 - step : step;
        for (int kk = 0; kk < c->ncol; ++kk) {
            int k = reverse ? c->ncol - 1 - kk : kk;
            int colour = c->ncol == 2 ? k : -1;
            const T *lam = v.lam + (int64_t)lv * lam_step(L);
            T *dst = inpl ? cur : other;  // snapshot semantics unless colour steps may run in place
            if (L.bs > 1) CSX_TRY(launch_block_sweep<T>(L, v.A, lam, b, cur, dst, colour, reverse, xzero, s));
            else CSX_TRY(launch_sweep<T>(L, v.A, lam, b, cur, dst, colour, xzero, s));
            if (!inpl) std::swap(cur, other);
            xzero = false;
        }
    }
    return CS_OK;
}

template <typename T>
static int out_of_place_steps(const cs_cascade *c, const Level &L) {
    return inplace_colours(c, L) ? 0 : c->nu * c->ncol;
}

template <typename T>
static cs_status coarse_solve_t(const cs_hierarchy *h, const T *b, T *x, cudaStream_t s);
template <>
cs_status coarse_solve_t<double>(const cs_hierarchy *h, const double *b, double *x, cudaStream_t s) {
    return launch_coarse_solve(h, b, x, s);
}
template <>
cs_status coarse_solve_t<float>(const cs_hierarchy *h, const float *b, float *x, cudaStream_t s) {
    return launch_coarse_solve32(h, b, x, s);
}
template <>
cs_status coarse_solve_t<__nv_bfloat16>(const cs_hierarchy *h, const __nv_bfloat16 *b, __nv_bfloat16 *x,
                                        cudaStream_t s) {
    return launch_coarse_solve16(h, b, x, s);
}

// zero-initial-guess cycle on level l: reads v.b, leaves the result in v.x
template <typename T>
static cs_status v0_enqueue(const cs_hierarchy *h, const cs_cascade *c, int l, int order, int mu_pre, int mu_post,
                            cudaStream_t s) {
    View<T> v = view<T>(h, c, l);
    if (l == h->nlev - 1) return coarse_solve_t<T>(h, v.b, v.x, s);
    const Level &L = h->lev[l];
    const Level &Lc = h->lev[l + 1];
    View<T> vc = view<T>(h, c, l + 1);
    T *cur = v.x, *other = v.t;
    bool xzero = true;
    for (int m = 0; m < mu_pre; ++m)
        CSX_TRY(smooth_apply<T>(h, c, l, v, v.b, cur, other, order == CS_RF, xzero, s));
    if (xzero) {
        CSX_CUDA(cudaMemsetAsync(cur, 0, sizeof(T) * L.g.N, s));
        xzero = false;
    }
    CSX_TRY(launch_residual_restrict<T>(L, Lc, v.A, v.b, cur, vc.b, other, s));  // other: free until prolongation
    CSX_TRY(v0_enqueue<T>(h, c, l + 1, order, mu_pre, mu_post, s));
    int P = mu_post * out_of_place_steps<T>(c, L);
    T *out = (P % 2 == 0) ? v.x : v.t;
    CSX_TRY(launch_prolong_correct<T>(L, Lc, vc.x, cur, out, s));
    cur = out;
    other = (out == v.x) ? v.t : v.x;
    for (int m = 0; m < mu_post; ++m)
        CSX_TRY(smooth_apply<T>(h, c, l, v, v.b, cur, other, false, xzero, s));
    if (cur != v.x) {
        set_error("internal: V-cycle result not in place");
        return CS_ERR_ARG;
    }
    return CS_OK;
}

// Launch the captured zero-guess cycle for these options (capturing it on
// first use): reads level-0 b (FP64 or FP32 state), writes level-0 x.
static cs_status run_v0(const cs_hierarchy *h, cs_cascade *c, const cs_vcycle_opts &o, cudaStream_t s) {
    for (auto &g : c->graphs)
        if (g.prec == o.precision && g.order == o.order && g.mu_pre == o.mu_pre && g.mu_post == o.mu_post) {
            CSX_CUDA(cudaGraphLaunch(g.exec, s));
            count_launch(g.kernels);
            return CS_OK;
        }
    // capture after the work already queued on s (the capture stream is separate)
    cudaStream_t cs = c->capture_stream;
    CSX_CUDA(cudaStreamSynchronize(s));
    CSX_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const int64_t before = g_launches.load();
    cs_status rc = o.precision == CS_FP32   ? v0_enqueue<float>(h, c, 0, o.order, o.mu_pre, o.mu_post, cs)
                   : o.precision == CS_BF16 ? v0_enqueue<__nv_bfloat16>(h, c, 0, o.order, o.mu_pre, o.mu_post, cs)
                                            : v0_enqueue<double>(h, c, 0, o.order, o.mu_pre, o.mu_post, cs);
    const int64_t kernels = g_launches.load() - before;  // recorded, not executed
    g_launches.fetch_sub(kernels);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (rc != CS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    c->graphs.push_back({o.precision, o.order, o.mu_pre, o.mu_post, exec, kernels});
    CSX_CUDA(cudaGraphLaunch(exec, s));
    count_launch(kernels);
    return CS_OK;
}

static cs_status check_cycle_opts(const cs_hierarchy *h, const cs_cascade *c, const cs_vcycle_opts *o) {
    if (!o || o->mu_pre < 0 || o->mu_post < 0 || o->mu_pre > 16 || o->mu_post > 16 ||
        (o->order != CS_RF && o->order != CS_FF) ||
        (o->precision != CS_FP64 && o->precision != CS_FP32 && o->precision != CS_BF16)) {
        set_error("invalid V-cycle options");
        return CS_ERR_ARG;
    }
    if (o->precision == CS_FP32 && !c->lowp) {
        set_error("FP32 cycles need a cascade built with lowp = 1");
        return CS_ERR_ARG;
    }
    if (o->precision == CS_BF16 && c->lo16.empty()) {
        set_error("BF16 cycles need a cascade built with lowp = 2");
        return CS_ERR_ARG;
    }
    if (h->cn == 0) {
        set_error("the hierarchy has no coarsest-level factorisation (periodic, or coarsest level too large)");
        return CS_ERR_UNSUPPORTED;
    }
    return CS_OK;
}

static double host_sum(const cs_hierarchy *h, int nred, cudaStream_t s, cs_status *rc) {
    *rc = launch_finish_sum(h->red, nred, s);
    if (*rc != CS_OK) return 0.0;
    cudaError_t e = cudaMemcpyAsync(h->red_host, h->red + nred, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *rc = cuda_fail(e, "reduction readback", __FILE__, __LINE__);
        return 0.0;
    }
    return h->red_host[0];
}

static int residual_blocks(const Level &L) {
    dim3 g = node_grid(L.g);
    return (int)(g.x * g.y * g.z);
}

}  // namespace csx

using namespace csx;

extern "C" {

const char *cs_last_error(void) { return g_err.c_str(); }

cs_status cs_setup_hierarchy(const cs_stencil *A0, const cs_hierarchy_opts *opts_in, cs_stream stream,
                             cs_hierarchy **out) {
    if (!A0 || !out) { set_error("null argument"); return CS_ERR_ARG; }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    cs_hierarchy_opts opts{4, 0, 1, 0};
    if (opts_in) opts = *opts_in;
    if (opts.coarse_max <= 0) opts.coarse_max = 4;
    if (opts.block == 0) opts.block = 1;
    int dim = A0->dim;
    if (dim != 2 && dim != 3) { set_error("dim must be 2 or 3"); return CS_ERR_ARG; }
    int n[3] = {A0->n[0], A0->n[1], dim == 3 ? A0->n[2] : 1};
    if (n[0] < 1 || n[1] < 1 || n[2] < 1 || (dim == 2 && A0->n[2] > 1)) { set_error("bad grid size"); return CS_ERR_ARG; }
    if ((int64_t)n[0] * n[1] * n[2] >= (int64_t)1 << 31) { set_error("grid too large (N must fit in 31 bits)"); return CS_ERR_ARG; }
    if (A0->nst < 1 || A0->nst > 27 || !A0->coeff) { set_error("bad stencil"); return CS_ERR_ARG; }
    if (opts.block < 1 || opts.block > (dim == 3 ? 2 : 3)) {
        set_error("block edge must be 1..%d in %dD", dim == 3 ? 2 : 3, dim);
        return CS_ERR_UNSUPPORTED;
    }
    bool star = true, centre = false;
    bool seen[27] = {false};
    for (int s2 = 0; s2 < A0->nst; ++s2) {
        const int *o = A0->off[s2];
        for (int d = 0; d < 3; ++d)
            if (o[d] < -1 || o[d] > 1) { set_error("stencil offsets must lie in {-1,0,1}"); return CS_ERR_ARG; }
        if (dim == 2 && o[2] != 0) { set_error("2D stencil with a z offset"); return CS_ERR_ARG; }
        int b = box_slot(dim, o);
        if (seen[b]) { set_error("duplicate stencil offset"); return CS_ERR_ARG; }
        seen[b] = true;
        if (o[0] == 0 && o[1] == 0 && o[2] == 0) centre = true;
        if (!is_star_offset(dim, o)) star = false;
    }
    if (!centre) { set_error("stencil needs the (0,0,0) entry"); return CS_ERR_ARG; }
    if (A0->periodic && opts.max_levels != 1) {
        set_error("periodic operators are accepted only with max_levels = 1");
        return CS_ERR_UNSUPPORTED;
    }

    cs_hierarchy *h = new cs_hierarchy();
    h->dim = dim;
    h->periodic = A0->periodic != 0;
    cs_status rc = CS_OK;
    {
        Level L0;
        L0.g = make_grid(dim, n[0], n[1], n[2]);
        L0.kind = star ? STAR : BOX;
        set_blocks(L0, opts.block);
        L0.nst = star ? 2 * dim + 1 : (dim == 3 ? 27 : 9);
        fill_offsets(L0);
        if ((rc = dalloc_t(&L0.A, (size_t)L0.nst * L0.g.N, &h->bytes, s)) != CS_OK) goto fail_nolevel;
        h->lev.push_back(L0);
        Level &L = h->lev[0];
        cudaError_t e = cudaMemsetAsync(L.A, 0, sizeof(double) * L.nst * L.g.N, s);
        for (int s2 = 0; s2 < A0->nst && e == cudaSuccess; ++s2) {
            int slot = star ? star_slot(A0->off[s2]) : box_slot(dim, A0->off[s2]);
            e = cudaMemcpyAsync(L.A + (int64_t)slot * L.g.N, A0->coeff + (int64_t)s2 * L.g.N, sizeof(double) * L.g.N,
                                A0->coeff_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
        }
        if (A0->coeff_on_host && e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "copy operator", __FILE__, __LINE__); goto fail; }
        if (!h->periodic && (rc = drop_outside_couplings(L, s)) != CS_OK) goto fail;
        if (!opts.no_reuse && (rc = level_margin(L, h->periodic, s)) != CS_OK) goto fail;
        if (!h->periodic && (rc = check_symmetric(L, s)) != CS_OK) goto fail;
    }
    while (!h->periodic && (opts.max_levels <= 0 || (int)h->lev.size() < opts.max_levels)) {
        const Level &F = h->lev.back();
        int mx = std::max(F.g.nx, std::max(F.g.ny, dim == 3 ? F.g.nz : 0));
        int mn = std::min(F.g.nx, std::min(F.g.ny, dim == 3 ? F.g.nz : F.g.ny));
        if (mx <= opts.coarse_max || mn < 2) break;
        Level C;
        C.g = make_grid(dim, F.g.nx / 2, F.g.ny / 2, dim == 3 ? F.g.nz / 2 : 1);
        C.kind = BOX;
        set_blocks(C, opts.block);
        C.nst = dim == 3 ? 27 : 9;
        fill_offsets(C);
        if ((rc = dalloc_t(&C.A, (size_t)C.nst * C.g.N, &h->bytes, s)) != CS_OK) goto fail;
        h->lev.push_back(C);
        if ((rc = galerkin_level(h->lev[h->lev.size() - 2], h->lev.back(), !opts.no_reuse, s)) != CS_OK) goto fail;
        if ((rc = check_symmetric(h->lev.back(), s)) != CS_OK) goto fail;
        if (!opts.no_reuse && (rc = level_margin(h->lev.back(), false, s)) != CS_OK) goto fail;
    }
    h->nlev = (int)h->lev.size();
    for (auto &L : h->lev) {
        if ((rc = dalloc_t(&L.b, L.g.N, &h->bytes, s)) != CS_OK) goto fail;
        if ((rc = dalloc_t(&L.x, L.g.N, &h->bytes, s)) != CS_OK) goto fail;
        if ((rc = dalloc_t(&L.t, L.g.N, &h->bytes, s)) != CS_OK) goto fail;
    }
    {
        int nred = std::max(residual_blocks(h->lev[0]), NRED);
        if ((rc = dalloc_t(&h->red, (size_t)nred + 8, &h->bytes, s)) != CS_OK) goto fail;
        cudaError_t e = cudaMallocHost(&h->red_host, 64 * sizeof(double));
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMallocHost", __FILE__, __LINE__); goto fail; }
        if ((rc = dalloc_t(&h->hb, h->lev[0].g.N, &h->bytes, s)) != CS_OK) goto fail;
        if ((rc = dalloc_t(&h->hx, h->lev[0].g.N, &h->bytes, s)) != CS_OK) goto fail;
    }
    // the dense factorisation runs in one CTA (O(n^3) FP64 operations): up to
    // 1024 unknowns; a larger coarsest level (a hierarchy cut short by
    // max_levels, kept for its cascade setup) is not factorised and cycles on
    // it report CS_ERR_UNSUPPORTED
    if (!h->periodic && h->lev.back().g.N <= 1024) {
        if ((rc = coarse_factor(h, s)) != CS_OK) goto fail;
    }
    {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "hierarchy setup", __FILE__, __LINE__); goto fail; }
    }
    *out = h;
    return CS_OK;
fail:
fail_nolevel:
    cs_destroy_hierarchy(h);
    return rc;
}

void cs_destroy_hierarchy(cs_hierarchy *h) {
    if (!h) return;
    for (auto &L : h->lev) { dfree(L.A); dfree(L.b); dfree(L.x); dfree(L.t); }
    dfree(h->cinv); dfree(h->red); dfree(h->hb); dfree(h->hx); dfree(h->fine_r);
    if (h->red_host) cudaFreeHost(h->red_host);
    delete h;
}

int64_t cs_hierarchy_bytes(const cs_hierarchy *h) { return h ? h->bytes : 0; }
int64_t cs_cascade_bytes(const cs_cascade *c) { return c ? c->bytes : 0; }

cs_status cs_setup_cascade(cs_hierarchy *h, const cs_cascade_opts *o, cs_stream stream, cs_cascade **out) {
    if (!h || !o || !out) { set_error("null argument"); return CS_ERR_ARG; }
    *out = nullptr;
    if (o->kind != CS_ADDITIVE && o->kind != CS_MULTIPLICATIVE) { set_error("bad cascade kind"); return CS_ERR_ARG; }
    if (o->nu < 1 || o->nu > 8) { set_error("nu must be in 1..8"); return CS_ERR_ARG; }
    if (o->alpha < 0) { set_error("alpha must be >= 0 (0: no truncation)"); return CS_ERR_ARG; }
    if (o->alpha > 0 && o->model) {
        set_error("truncation does not combine with the learned setup");
        return CS_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cs_cascade *c = new cs_cascade();
    c->h = h;
    c->kind = o->kind;
    c->nu = o->nu;
    c->ncol = o->kind == CS_MULTIPLICATIVE ? 2 : 1;
    c->nlev = h->nlev > 1 ? h->nlev - 1 : 1;
    c->lowp = o->lowp != 0;
    if (o->lowp < 0 || o->lowp > 2) { set_error("lowp must be 0, 1 or 2"); delete c; return CS_ERR_ARG; }
    if (o->setup_precision != CS_FP64 && o->setup_precision != CS_FP32) {
        set_error("setup_precision must be CS_FP64 or CS_FP32");
        delete c;
        return CS_ERR_ARG;
    }
    if (o->setup_precision == CS_FP32) {
        // truncation ranks columns by norm: FP32 products would flip near ties
        if (o->model || o->alpha > 0) {
            set_error("the FP32 setup takes no model and no truncation");
            delete c;
            return CS_ERR_UNSUPPORTED;
        }
    }
    if (o->sketch < 0 || o->sketch > 128) {
        set_error("sketch must be in 0..128 (0: the exact setup)");
        delete c;
        return CS_ERR_ARG;
    }
    if (o->sketch > 0) {
        bool blocks = false;
        for (int l = 0; l < h->nlev; ++l) blocks = blocks || h->lev[l].bs > 1;
        if (blocks || o->model || o->alpha > 0 || h->periodic) {
            set_error("the sketched setup is implemented for Dirichlet point-block hierarchies without truncation "
                      "or a model");
            delete c;
            return CS_ERR_UNSUPPORTED;
        }
    }
    if (o->lowp == 2)
        for (int l = 0; l < h->nlev; ++l)
            if (h->lev[l].bs > 1) {
                set_error("BF16 copies (lowp = 2) are implemented for point-block hierarchies only");
                delete c;
                return CS_ERR_UNSUPPORTED;
            }
    cs_status rc = CS_OK;
    c->lam.assign(c->nlev, nullptr);
    for (int l = 0; l < c->nlev; ++l)
        if ((rc = dalloc_t(&c->lam[l], (size_t)c->nu * lam_step(h->lev[l]), &c->bytes, s)) != CS_OK) goto fail;
    {
        // The levels' setups are independent of one another.  The coarse levels
        // (small, latency-bound kernels) run concurrently, each from its own host
        // thread on its own stream, while the finest level runs here on s.
        auto level_setup = [&](int l, cudaStream_t st) -> cs_status {
            const Level &L = h->lev[l];
            if (o->sketch > 0)
                return cascade_setup_level_sketch(h, l, c->kind, c->nu, o->prescale, o->sketch, o->sketch_seed,
                                                  o->sketch_exact_first, o->setup_precision == CS_FP32, c->lam[l], st);
            if (L.bs > 1)
                return cascade_setup_level_blocks(h, l, c->kind, c->nu, o->prescale, o->alpha,
                                                  o->setup_precision == CS_FP32, c->lam[l], st);
            int64_t peak = 0;
            return cascade_setup_level(h, l, c->kind, c->nu, o->prescale, !o->no_reuse, o->alpha,
                                       o->setup_precision == CS_FP32, c->lam[l], st, &peak);
        };
        auto finest = [&]() -> cs_status {
            const Level &L = h->lev[0];
            if (o->model) {
                if (L.bs < 2 || L.g.dim != 2 || c->kind != CS_ADDITIVE) {
                    set_error("the learned setup needs an additive cascade on a 2D block level");
                    return CS_ERR_UNSUPPORTED;
                }
                // exact level-1 blocks (one least-squares problem per block) are the yardstick of the prediction
                double *lam1 = nullptr;
                cs_status r = dalloc_t(&lam1, (size_t)lam_step(L), nullptr, s);
                if (r != CS_OK) return r;
                r = cascade_setup_level_blocks(h, 0, CS_ADDITIVE, 1, o->prescale, 0, false, lam1, s);
                if (r == CS_OK)
                    r = learned_setup_level0(h, c, const_cast<cs_mlp *>(o->model), o->model_tol > 0 ? o->model_tol : 0.05,
                                             c->lam[0], lam1, s);
                dfree(lam1, s);
                if (r != CS_OK) return r;
                // no block kept its prediction: the exact setup of the whole level
                c->learned_used = c->learned_accepted > 0 ? 1 : 0;
                if (c->learned_used) return CS_OK;
            }
            return level_setup(0, s);
        };
        // inside cs_setup_many's workers (already one thread per problem) the
        // levels run one after another on s
        const int nco = g_serial_levels ? 0 : c->nlev - 1;
        std::vector<cudaStream_t> ls(nco, nullptr);
        std::vector<cudaEvent_t> ev(nco + 1, nullptr);
        std::vector<cs_status> lrc(nco, CS_OK);
        std::vector<std::string> lmsg(nco);
        std::vector<std::thread> th;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
        for (int k = 0; k < nco && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&ls[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev[k + 1], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ls[k], ev[0], 0);
        }
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cascade setup streams", __FILE__, __LINE__);
        } else {
            for (int k = 0; k < nco; ++k)
                th.emplace_back([&, k] {
                    cudaError_t te = cudaSetDevice(dev);
                    lrc[k] = te == cudaSuccess ? level_setup(k + 1, ls[k]) : cuda_fail(te, "set device", __FILE__, __LINE__);
                    if (lrc[k] != CS_OK) lmsg[k] = cs_last_error();
                    cudaEventRecord(ev[k + 1], ls[k]);
                });
            rc = finest();
            for (int l = nco + 1; l < c->nlev && rc == CS_OK; ++l) rc = level_setup(l, s);
            for (auto &t : th) t.join();
            for (int k = 0; k < nco; ++k) {
                if (rc == CS_OK && lrc[k] != CS_OK) { rc = lrc[k]; set_error("%s", lmsg[k].c_str()); }
                cudaStreamWaitEvent(s, ev[k + 1], 0);
            }
        }
        for (int k = 0; k < nco; ++k) {
            if (ls[k]) {
                if (rc != CS_OK) cudaStreamSynchronize(ls[k]);
                cudaStreamDestroy(ls[k]);
            }
        }
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        if (rc != CS_OK) {
            cudaStreamSynchronize(s);
            goto fail;
        }
    }
    if (c->lowp) {
        c->lo.resize(h->nlev);
        for (int l = 0; l < h->nlev; ++l) {
            const Level &L = h->lev[l];
            LowLevel &lo = c->lo[l];
            const int64_t N = L.g.N;
            if ((rc = dalloc_t(&lo.A, (size_t)lo_nst(L) * N, &c->bytes, s)) != CS_OK) goto fail;
            if (L.sym32) {
                if ((rc = launch_copy_box_sym32(L, lo.A, s)) != CS_OK) goto fail;
            } else if ((rc = launch_copy_d2f((int64_t)L.nst * N, L.A, lo.A, s)) != CS_OK) {
                goto fail;
            }
            if (l < c->nlev) {
                if ((rc = dalloc_t(&lo.lam, (size_t)c->nu * lam_step(L), &c->bytes, s)) != CS_OK) goto fail;
                if ((rc = launch_copy_d2f((int64_t)c->nu * lam_step(L), c->lam[l], lo.lam, s)) != CS_OK) goto fail;
            }
            if ((rc = dalloc_t(&lo.b, N, &c->bytes, s)) != CS_OK) goto fail;
            if ((rc = dalloc_t(&lo.x, N, &c->bytes, s)) != CS_OK) goto fail;
            if ((rc = dalloc_t(&lo.t, N, &c->bytes, s)) != CS_OK) goto fail;
        }
    }
    if (o->lowp == 2) {  // BF16 storage of operators, Lambda and vectors (FP32 arithmetic)
        c->lo16.resize(h->nlev);
        for (int l = 0; l < h->nlev; ++l) {
            const Level &L = h->lev[l];
            LowLevel16 &lo = c->lo16[l];
            const int64_t N = L.g.N;
            if ((rc = dalloc_t(&lo.A, (size_t)L.nst * N, &c->bytes, s)) != CS_OK) goto fail;
            if ((rc = launch_copy_d2bf((int64_t)L.nst * N, L.A, lo.A, s)) != CS_OK) goto fail;
            if (l < c->nlev) {
                if ((rc = dalloc_t(&lo.lam, (size_t)c->nu * lam_step(L), &c->bytes, s)) != CS_OK) goto fail;
                if ((rc = launch_copy_d2bf((int64_t)c->nu * lam_step(L), c->lam[l], lo.lam, s)) != CS_OK) goto fail;
            }
            if ((rc = dalloc_t(&lo.b, N, &c->bytes, s)) != CS_OK) goto fail;
            if ((rc = dalloc_t(&lo.x, N, &c->bytes, s)) != CS_OK) goto fail;
            if ((rc = dalloc_t(&lo.t, N, &c->bytes, s)) != CS_OK) goto fail;
        }
    }
    {
        cudaError_t e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cascade setup", __FILE__, __LINE__); goto fail; }
    }
    *out = c;
    return CS_OK;
fail:
    cs_destroy_cascade(c);
    return rc;
}

cs_status cs_setup_many(int nprob, const cs_stencil *A, const cs_hierarchy_opts *ho, const cs_cascade_opts *co,
                        int nthreads, cs_stream stream, cs_hierarchy **h, cs_cascade **c) {
    if (nprob < 0 || (nprob > 0 && (!A || !ho || !co || !h || !c))) { set_error("null argument"); return CS_ERR_ARG; }
    for (int p = 0; p < nprob; ++p) { h[p] = nullptr; c[p] = nullptr; }
    if (nprob == 0) return CS_OK;
    if (nthreads <= 0) nthreads = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    nthreads = std::min(nthreads, nprob);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    CSX_CUDA(cudaGetDevice(&dev));
    cudaEvent_t ready = nullptr;
    CSX_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ready, s);
    if (e != cudaSuccess) { cudaEventDestroy(ready); return cuda_fail(e, "setup many", __FILE__, __LINE__); }
    std::vector<cs_status> prc(nprob, CS_OK);
    std::vector<std::string> pmsg(nprob);
    std::vector<cudaStream_t> ws(nthreads, nullptr);
    std::vector<cudaEvent_t> wd(nthreads, nullptr);
    std::vector<std::thread> th;
    for (int k = 0; k < nthreads; ++k)
        th.emplace_back([&, k] {
            g_serial_levels = true;
            cudaError_t te = cudaSetDevice(dev);
            if (te == cudaSuccess) te = cudaStreamCreateWithFlags(&ws[k], cudaStreamNonBlocking);
            if (te == cudaSuccess) te = cudaEventCreateWithFlags(&wd[k], cudaEventDisableTiming);
            if (te == cudaSuccess) te = cudaStreamWaitEvent(ws[k], ready, 0);
            for (int p = k; p < nprob; p += nthreads) {
                if (te != cudaSuccess) {
                    prc[p] = cuda_fail(te, "setup worker", __FILE__, __LINE__);
                } else {
                    prc[p] = cs_setup_hierarchy(&A[p], ho, ws[k], &h[p]);
                    if (prc[p] == CS_OK) prc[p] = cs_setup_cascade(h[p], co, ws[k], &c[p]);
                }
                if (prc[p] != CS_OK) pmsg[p] = cs_last_error();
            }
            if (wd[k]) cudaEventRecord(wd[k], ws[k]);
        });
    for (auto &t : th) t.join();
    cs_status rc = CS_OK;
    for (int p = 0; p < nprob && rc == CS_OK; ++p)
        if (prc[p] != CS_OK) {
            rc = prc[p];
            set_error("problem %d: %s", p, pmsg[p].c_str());
        }
    for (int k = 0; k < nthreads; ++k) {
        if (wd[k]) { cudaStreamWaitEvent(s, wd[k], 0); cudaEventDestroy(wd[k]); }
        if (ws[k]) { if (rc != CS_OK) cudaStreamSynchronize(ws[k]); cudaStreamDestroy(ws[k]); }
    }
    cudaEventDestroy(ready);
    if (rc != CS_OK) {
        cudaStreamSynchronize(s);
        for (int p = 0; p < nprob; ++p) {
            cs_destroy_cascade(c[p]);
            cs_destroy_hierarchy(h[p]);
            c[p] = nullptr;
            h[p] = nullptr;
        }
    }
    return rc;
}

void cs_destroy_cascade(cs_cascade *c) {
    if (!c) return;
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    for (double *p : c->lam) dfree(p);
    for (auto &lo : c->lo) { dfree(lo.A); dfree(lo.lam); dfree(lo.b); dfree(lo.x); dfree(lo.t); }
    for (auto &lo : c->lo16) { dfree(lo.A); dfree(lo.lam); dfree(lo.b); dfree(lo.x); dfree(lo.t); }
    dfree(c->fine_b32); dfree(c->fine_x32); dfree(c->gm_V); dfree(c->gm_h); dfree(c->gm_Z);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
}

cs_status cs_vcycle(const cs_hierarchy *h, cs_cascade *c, const cs_vcycle_opts *o, const double *b, double *x,
                    cs_stream stream) {
    if (!h || !c || !b || !x) { set_error("null argument"); return CS_ERR_ARG; }
    CSX_TRY(check_cycle_opts(h, c, o));
    cudaStream_t s = (cudaStream_t)stream;
    const Level &L = h->lev[0];
    if (o->precision == CS_FP32) {
        CSX_TRY(launch_residual64(L, L.A, b, x, nullptr, c->lo[0].b, nullptr, 0, s));
        CSX_TRY(run_v0(h, c, *o, s));
        CSX_TRY(launch_axpy_f32(L.g.N, c->lo[0].x, x, s));
    } else if (o->precision == CS_BF16) {
        CSX_TRY(launch_residual64_bf16(L, L.A, b, x, c->lo16[0].b, s));
        CSX_TRY(run_v0(h, c, *o, s));
        CSX_TRY(launch_axpy_bf16(L.g.N, c->lo16[0].x, x, s));
    } else {
        CSX_TRY(launch_residual64(L, L.A, b, x, L.b, nullptr, nullptr, 0, s));
        CSX_TRY(run_v0(h, c, *o, s));
        CSX_TRY(launch_add64(L.g.N, L.x, x, s));
    }
    return CS_OK;
}

cs_status cs_smooth(const cs_hierarchy *h, cs_cascade *c, int level, int reverse, const double *b, double *x,
                    cs_stream stream) {
    if (!h || !c || !b || !x) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= c->nlev) { set_error("level %d has no smoother", level); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    View<double> v = view<double>(h, c, level);
    double *cur = x, *other = h->lev[level].t;
    bool xzero = false;
    CSX_TRY(smooth_apply<double>(h, c, level, v, b, cur, other, reverse != 0, xzero, s));
    if (cur != x) CSX_CUDA(cudaMemcpyAsync(x, cur, sizeof(double) * h->lev[level].g.N, cudaMemcpyDeviceToDevice, s));
    return CS_OK;
}

cs_status cs_sweep(const cs_hierarchy *h, cs_cascade *c, int level, int step, int colour, int precision,
                   const void *b, const void *x, void *out, cs_stream stream) {
    if (!h || !c || !b || !x || !out) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= c->nlev) { set_error("level %d has no smoother", level); return CS_ERR_ARG; }
    if (step < 0 || step >= c->nu) { set_error("step out of range"); return CS_ERR_ARG; }
    if (colour < -1 || colour > 1 || (colour >= 0 && c->ncol != 2) || (colour < 0 && c->ncol != 1)) {
        set_error("colour does not match the cascade kind");
        return CS_ERR_ARG;
    }
    const Level &L = h->lev[level];
    if (out == x && !(colour >= 0 && L.kind == STAR)) {
        set_error("out may alias x only for a colour step on a 5/7-point level");
        return CS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t st = (int64_t)step * lam_step(L);
    if (precision == CS_FP32) {
        if (!c->lowp) { set_error("FP32 steps need lowp"); return CS_ERR_ARG; }
        const LowLevel &lo = c->lo[level];
        if (L.bs > 1)
            return launch_block_sweep<float>(L, lo.A, lo.lam + st, (const float *)b, (const float *)x, (float *)out,
                                             colour, false, false, s);
        return launch_sweep<float>(L, lo.A, lo.lam + st, (const float *)b, (const float *)x, (float *)out, colour,
                                   false, s);
    }
    if (precision == CS_BF16) {
        if (c->lo16.empty()) { set_error("BF16 steps need lowp = 2"); return CS_ERR_ARG; }
        const LowLevel16 &lo = c->lo16[level];
        return launch_sweep<__nv_bfloat16>(L, lo.A, lo.lam + st, (const __nv_bfloat16 *)b, (const __nv_bfloat16 *)x,
                                           (__nv_bfloat16 *)out, colour, false, s);
    }
    if (precision != CS_FP64) { set_error("bad precision"); return CS_ERR_ARG; }
    if (L.bs > 1)
        return launch_block_sweep<double>(L, L.A, c->lam[level] + st, (const double *)b, (const double *)x,
                                          (double *)out, colour, false, false, s);
    return launch_sweep<double>(L, L.A, c->lam[level] + st, (const double *)b, (const double *)x, (double *)out,
                                colour, false, s);
}

cs_status cs_sweep_rhs(const cs_hierarchy *h, cs_cascade *c, int level, int step, int colour, int transpose,
                       int precision, int nrhs, const void *b, const void *x, void *out, cs_stream stream) {
    if (!h || !c || !b || !x || !out) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= c->nlev) { set_error("level %d has no smoother", level); return CS_ERR_ARG; }
    if (step < 0 || step >= c->nu) { set_error("step out of range"); return CS_ERR_ARG; }
    if (nrhs < 1 || nrhs > 32) { set_error("nrhs must be in 1..32"); return CS_ERR_ARG; }
    if (colour < -1 || colour > 1 || (colour >= 0 && c->ncol != 2) || (colour < 0 && c->ncol != 1)) {
        set_error("colour does not match the cascade kind");
        return CS_ERR_ARG;
    }
    const Level &L = h->lev[level];
    if (out == x && !(colour >= 0 && L.kind == STAR)) {
        set_error("out may alias x only for a colour step on a 5/7-point level");
        return CS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t st = (int64_t)step * lam_step(L);
    if (precision == CS_FP32) {
        if (!c->lowp) { set_error("FP32 steps need lowp"); return CS_ERR_ARG; }
        const LowLevel &lo = c->lo[level];
        if (L.sym32) {
            set_error("FP32 multi-RHS steps on a 3D 27-point level with symmetric FP32 storage are not implemented");
            return CS_ERR_UNSUPPORTED;
        }
        return launch_block_sweep_m<float>(L, lo.A, lo.lam + st, (const float *)b, (const float *)x, (float *)out,
                                           nrhs, colour, transpose != 0, s);
    }
    if (precision != CS_FP64) { set_error("bad precision"); return CS_ERR_ARG; }
    return launch_block_sweep_m<double>(L, L.A, c->lam[level] + st, (const double *)b, (const double *)x,
                                        (double *)out, nrhs, colour, transpose != 0, s);
}

int64_t cs_kernel_launches(void) { return g_launches.load(); }

cs_status cs_learned_status(const cs_cascade *c, int *used, double *ratio) {
    if (!c) { set_error("null argument"); return CS_ERR_ARG; }
    if (used) *used = c->learned_used;
    if (ratio) *ratio = c->learned_ratio;
    return CS_OK;
}

cs_status cs_learned_stats(const cs_cascade *c, int64_t *blocks, int64_t *full_blocks, int64_t *predicted_blocks,
                           double *ratio_predicted, double *ratio_used) {
    if (!c) { set_error("null argument"); return CS_ERR_ARG; }
    if (blocks) *blocks = c->learned_blocks;
    if (full_blocks) *full_blocks = c->learned_full;
    if (predicted_blocks) *predicted_blocks = c->learned_used == 1 ? c->learned_accepted : 0;
    if (ratio_predicted) *ratio_predicted = c->learned_ratio;
    if (ratio_used) *ratio_used = c->learned_used == 1 ? c->learned_ratio_used : 1.0;
    return CS_OK;
}

cs_status cs_residual_restrict(const cs_hierarchy *h, int level, const double *b, const double *x, double *rc,
                               cs_stream stream) {
    if (!h || !b || !x || !rc) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level + 1 >= h->nlev) { set_error("level %d has no coarser level", level); return CS_ERR_ARG; }
    return launch_residual_restrict<double>(h->lev[level], h->lev[level + 1], h->lev[level].A, b, x, rc,
                                            h->lev[level].t, (cudaStream_t)stream);
}

cs_status cs_prolong_correct(const cs_hierarchy *h, int level, const double *xc, double *x, cs_stream stream) {
    if (!h || !xc || !x) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level + 1 >= h->nlev) { set_error("level %d has no coarser level", level); return CS_ERR_ARG; }
    return launch_prolong_correct<double>(h->lev[level], h->lev[level + 1], xc, x, x, (cudaStream_t)stream);
}

cs_status cs_residual_restrict_lowp(const cs_hierarchy *h, cs_cascade *c, int level, int precision, const void *b,
                                    const void *x, void *rc, cs_stream stream) {
    if (!h || !c || !b || !x || !rc) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level + 1 >= h->nlev) { set_error("level %d has no coarser level", level); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const Level &f = h->lev[level], &cl = h->lev[level + 1];
    if (precision == CS_FP32) {
        if (!c->lowp) { set_error("FP32 transfers need lowp"); return CS_ERR_ARG; }
        const LowLevel &lo = c->lo[level];
        return launch_residual_restrict<float>(f, cl, lo.A, (const float *)b, (const float *)x, (float *)rc, lo.t, s);
    }
    if (precision == CS_BF16) {
        if (c->lo16.empty()) { set_error("BF16 transfers need lowp = 2"); return CS_ERR_ARG; }
        const LowLevel16 &lo = c->lo16[level];
        return launch_residual_restrict<__nv_bfloat16>(f, cl, lo.A, (const __nv_bfloat16 *)b,
                                                       (const __nv_bfloat16 *)x, (__nv_bfloat16 *)rc, nullptr, s);
    }
    set_error("precision must be CS_FP32 or CS_BF16 (cs_residual_restrict takes FP64)");
    return CS_ERR_ARG;
}

cs_status cs_prolong_correct_lowp(const cs_hierarchy *h, cs_cascade *c, int level, int precision, const void *xc,
                                  void *x, cs_stream stream) {
    if (!h || !c || !xc || !x) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level + 1 >= h->nlev) { set_error("level %d has no coarser level", level); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const Level &f = h->lev[level], &cl = h->lev[level + 1];
    if (precision == CS_FP32) {
        if (!c->lowp) { set_error("FP32 transfers need lowp"); return CS_ERR_ARG; }
        return launch_prolong_correct<float>(f, cl, (const float *)xc, (const float *)x, (float *)x, s);
    }
    if (precision == CS_BF16) {
        if (c->lo16.empty()) { set_error("BF16 transfers need lowp = 2"); return CS_ERR_ARG; }
        return launch_prolong_correct<__nv_bfloat16>(f, cl, (const __nv_bfloat16 *)xc, (const __nv_bfloat16 *)x,
                                                     (__nv_bfloat16 *)x, s);
    }
    set_error("precision must be CS_FP32 or CS_BF16 (cs_prolong_correct takes FP64)");
    return CS_ERR_ARG;
}

cs_status cs_coarse_solve(const cs_hierarchy *h, const double *b, double *x, cs_stream stream) {
    if (!h || !b || !x) { set_error("null argument"); return CS_ERR_ARG; }
    if (h->cn == 0) { set_error("no coarsest-level factorisation"); return CS_ERR_UNSUPPORTED; }
    return launch_coarse_solve(h, b, x, (cudaStream_t)stream);
}

cs_status cs_residual(const cs_hierarchy *h, int level, const double *b, const double *x, double *r, double *norm2,
                      cs_stream stream) {
    if (!h || !b || !x || !r) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    const Level &L = h->lev[level];
    int nred = residual_blocks(L);
    bool want = norm2 != nullptr && level == 0;
    CSX_TRY(launch_residual64(L, L.A, b, x, r, nullptr, want ? h->red : nullptr, nred, s));
    if (norm2) {
        if (level != 0) {
            CSX_TRY(launch_dot(L.g.N, r, r, h->red, NRED, s));
            nred = NRED;
            cudaError_t e = cudaMemcpyAsync(h->red_host, h->red + nred, sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "norm readback", __FILE__, __LINE__);
            *norm2 = std::sqrt(h->red_host[0]);
        } else {
            cs_status rc;
            double v = host_sum(h, nred, s, &rc);
            if (rc != CS_OK) return rc;
            *norm2 = std::sqrt(v);
        }
    }
    return CS_OK;
}

static cs_status gmres(const cs_hierarchy *h, cs_cascade *c, const cs_solve_opts *o, const double *b, double *x,
                       double nb, cs_solve_info *info, cudaStream_t s);
static cs_status gmres_right(const cs_hierarchy *h, cs_cascade *c, const cs_solve_opts *o, const double *b,
                             double *x, double nb, cs_solve_info *info, cudaStream_t s);

cs_status cs_solve(const cs_hierarchy *h, cs_cascade *c, const cs_solve_opts *o_in, const double *b_in, double *x_in,
                   cs_solve_info *info, cs_stream stream) {
    if (!h || !c || !o_in || !b_in || !x_in) { set_error("null argument"); return CS_ERR_ARG; }
    cs_solve_opts o = *o_in;
    if (o.maxit <= 0) o.maxit = 100;
    if (o.tol <= 0) o.tol = 1e-10;
    if (o.restart <= 0) o.restart = 30;
    CSX_TRY(check_cycle_opts(h, c, &o.cycle));
    if (o.method != CS_STATIONARY && o.method != CS_GMRES && o.method != CS_REFINE && o.method != CS_GMRES_RIGHT) {
        set_error("bad solve method");
        return CS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const Level &L = h->lev[0];
    const int64_t N = L.g.N;
    const double *b = b_in;
    double *x = x_in;
    if (o.host_buffers) {
        CSX_CUDA(cudaMemcpyAsync(h->hb, b_in, sizeof(double) * N, cudaMemcpyHostToDevice, s));
        CSX_CUDA(cudaMemcpyAsync(h->hx, x_in, sizeof(double) * N, cudaMemcpyHostToDevice, s));
        b = h->hb;
        x = h->hx;
    }
    cs_solve_info inf{0, 0, 0.0, 0};
    cs_status rc = CS_OK;
    // ||b||
    CSX_TRY(launch_dot(N, b, b, h->red, NRED, s));
    CSX_CUDA(cudaMemcpyAsync(h->red_host, h->red + NRED, sizeof(double), cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaStreamSynchronize(s));
    double nb = std::sqrt(h->red_host[0]);
    if (nb == 0.0) {
        CSX_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, s));
        inf.converged = 1;
    } else if (o.method == CS_GMRES) {
        rc = gmres(h, c, &o, b, x, nb, &inf, s);
    } else if (o.method == CS_GMRES_RIGHT) {
        rc = gmres_right(h, c, &o, b, x, nb, &inf, s);
    } else {
        const bool lowp = o.cycle.precision == CS_FP32, bf16 = o.cycle.precision == CS_BF16;
        const int nred = residual_blocks(L);
        float *r32 = lowp ? c->lo[0].b : nullptr;
        double *r64 = lowp ? nullptr : L.b;  // FP64 cycles read it; BF16 cycles take a BF16 copy
        auto residual = [&]() -> cs_status {
            // with FP32 cycles the norm decides convergence only: block sums in FP32
            CSX_TRY(launch_residual64(L, L.A, b, x, r64, r32, h->red, nred, s, lowp));
            if (bf16) CSX_TRY(launch_copy_d2bf(N, L.b, c->lo16[0].b, s));
            return CS_OK;
        };
        CSX_TRY(residual());
        double rel = std::sqrt(host_sum(h, nred, s, &rc)) / nb;
        if (rc != CS_OK) return rc;
        const double rel0 = rel;
        if (o.hist && inf.nhist < o.hist_cap) o.hist[inf.nhist++] = rel;
        while (rel > o.tol && inf.iterations < o.maxit) {
            CSX_TRY(run_v0(h, c, o.cycle, s));
            if (lowp) CSX_TRY(launch_axpy_f32(N, c->lo[0].x, x, s));
            else if (bf16) CSX_TRY(launch_axpy_bf16(N, c->lo16[0].x, x, s));
            else CSX_TRY(launch_add64(N, L.x, x, s));
            ++inf.iterations;
            CSX_TRY(residual());
            rel = std::sqrt(host_sum(h, nred, s, &rc)) / nb;
            if (rc != CS_OK) return rc;
            if (o.hist && inf.nhist < o.hist_cap) o.hist[inf.nhist++] = rel;
            if (!std::isfinite(rel) || rel > 1e3 * std::max(rel0, 1.0)) {
                set_error("iteration diverged (relative residual %g)", rel);
                rc = CS_ERR_DIVERGED;
                break;
            }
        }
        inf.final_rel_residual = rel;
        inf.converged = rel <= o.tol;
        if (rc == CS_OK && !inf.converged) {
            set_error("not converged after %d iterations (relative residual %g)", inf.iterations, rel);
            rc = CS_ERR_NOTCONV;
        }
    }
    if (o.host_buffers) {
        CSX_CUDA(cudaMemcpyAsync(x_in, x, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
        CSX_CUDA(cudaStreamSynchronize(s));
    }
    if (info) *info = inf;
    return rc;
}

// Left-preconditioned restarted GMRES with M = V0 (the zero-initial-guess
// cycle), modified Gram-Schmidt and Givens rotations; the small Hessenberg
// problem is solved on the host.  Stops on the true relative residual.
static cs_status gmres(const cs_hierarchy *h, cs_cascade *c, const cs_solve_opts *o, const double *b, double *x,
                       double nb, cs_solve_info *inf, cudaStream_t s) {
    const Level &L = h->lev[0];
    const int64_t N = L.g.N;
    const int m = o->restart;
    const bool lowp = o->cycle.precision == CS_FP32, bf16 = o->cycle.precision == CS_BF16;
    if (c->gm_restart < m) {
        dfree(c->gm_V, s); dfree(c->gm_h, s);
        c->gm_V = nullptr; c->gm_h = nullptr;
        CSX_TRY(dalloc_t(&c->gm_V, (size_t)(m + 1) * N, &c->bytes, s));
        CSX_TRY(dalloc_t(&c->gm_h, (size_t)(m + 2) * 2, &c->bytes, s));
        c->gm_restart = m;
    }
    double *V = c->gm_V, *hd = c->gm_h;
    double *z = L.x;  // cycle output (FP64 path) / converted output (FP32 path)
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hh(m + 2);
    auto precond = [&](const double *rhs_dev) -> cs_status {
        // z = V0(rhs): rhs is in L.b (FP64) already, or converted for FP32
        if (lowp) {
            CSX_TRY(launch_copy_d2f(N, rhs_dev, c->lo[0].b, s));
            CSX_TRY(run_v0(h, c, o->cycle, s));
            CSX_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * N, s));
            CSX_TRY(launch_axpy_f32(N, c->lo[0].x, z, s));
        } else if (bf16) {
            CSX_TRY(launch_copy_d2bf(N, rhs_dev, c->lo16[0].b, s));
            CSX_TRY(run_v0(h, c, o->cycle, s));
            CSX_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * N, s));
            CSX_TRY(launch_axpy_bf16(N, c->lo16[0].x, z, s));
        } else {
            if (rhs_dev != L.b) CSX_CUDA(cudaMemcpyAsync(L.b, rhs_dev, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            CSX_TRY(run_v0(h, c, o->cycle, s));
        }
        return CS_OK;
    };
    auto dot_to = [&](const double *a, const double *bb, double *dst) -> cs_status {
        CSX_TRY(launch_dot(N, a, bb, h->red, NRED, s));
        CSX_CUDA(cudaMemcpyAsync(dst, h->red + NRED, sizeof(double), cudaMemcpyDeviceToDevice, s));
        return CS_OK;
    };
    // ||M b||
    CSX_TRY(precond(b));
    CSX_TRY(dot_to(z, z, hd));
    CSX_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double), cudaMemcpyDeviceToHost, s));
    CSX_CUDA(cudaStreamSynchronize(s));
    const double nmb = std::sqrt(hh[0]);
    const int nred = residual_blocks(L);
    double rel = 1.0;
    cs_status rc = CS_OK;
    for (;;) {
        CSX_TRY(launch_residual64(L, L.A, b, x, L.t, nullptr, h->red, nred, s));
        rel = std::sqrt(host_sum(h, nred, s, &rc)) / nb;
        if (rc != CS_OK) return rc;
        if (!std::isfinite(rel)) { set_error("GMRES diverged"); return CS_ERR_DIVERGED; }
        if (rel <= o->tol || inf->iterations >= o->maxit) break;
        CSX_TRY(precond(L.t));
        CSX_TRY(dot_to(z, z, hd));
        CSX_TRY(launch_scale_dev(N, hd, V, z, s));
        CSX_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double), cudaMemcpyDeviceToHost, s));
        CSX_CUDA(cudaStreamSynchronize(s));
        double beta = std::sqrt(hh[0]);
        if (inf->nhist == 0 && o->hist && inf->nhist < o->hist_cap) o->hist[inf->nhist++] = beta / nmb;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j;
        for (j = 0; j < m && inf->iterations < o->maxit; ++j) {
            CSX_TRY(launch_matvec64(L, L.A, V + (int64_t)j * N, L.b, s));
            CSX_TRY(precond(L.b));
            ++inf->iterations;
            for (int i = 0; i <= j; ++i) {
                CSX_TRY(dot_to(z, V + (int64_t)i * N, hd + i));
                CSX_TRY(launch_axpy_dev(N, hd + i, -1.0, V + (int64_t)i * N, z, s));
            }
            CSX_TRY(dot_to(z, z, hd + j + 1));
            CSX_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
            CSX_CUDA(cudaStreamSynchronize(s));
            double hn = std::sqrt(hh[j + 1]);
            if (hn > 0.0) CSX_TRY(launch_scale_dev(N, hd + j + 1, V + (int64_t)(j + 1) * N, z, s));
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i];
            H[(size_t)(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
            double d = std::sqrt(a * a + bb * bb);
            cs[j] = d > 0 ? a / d : 1.0;
            sn[j] = d > 0 ? bb / d : 0.0;
            H[(size_t)j * m + j] = d;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (o->hist && inf->nhist < o->hist_cap) o->hist[inf->nhist++] = std::fabs(g[j + 1]) / nmb;
            if (std::fabs(g[j + 1]) <= o->tol * nmb || hn == 0.0) { ++j; break; }
        }
        for (int i = j - 1; i >= 0; --i) {
            double sum = g[i];
            for (int k = i + 1; k < j; ++k) sum -= H[(size_t)i * m + k] * y[k];
            y[i] = sum / H[(size_t)i * m + i];
        }
        CSX_CUDA(cudaMemcpyAsync(hd, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
        CSX_TRY(launch_axpy_multi(N, j, hd, V, x, s));
        CSX_CUDA(cudaStreamSynchronize(s));  // y is a host buffer reused next restart
    }
    inf->final_rel_residual = rel;
    inf->converged = rel <= o->tol;
    if (!inf->converged) {
        set_error("GMRES not converged after %d iterations (relative residual %g)", inf->iterations, rel);
        return CS_ERR_NOTCONV;
    }
    return CS_OK;
}

// Right-preconditioned restarted GMRES in its flexible form: Z_j = M V_j is
// kept and x += Z y, with V an orthonormal (modified Gram-Schmidt) basis
// built from w = A Z_j.  With an FP64 cycle M is one fixed linear map and
// this is right-preconditioned GMRES (x_k minimises ||b - A x|| over
// x_0 + M K_k(A M, r_0)).  With FP32 / BF16 cycles M is that map only up to
// the cycle's rounding; keeping Z makes b - A x_k = V_{k+1}(beta e_1 - H y)
// hold up to FP64 rounding all the same, so the Givens estimate |g_{k+1}| is
// the true residual and the solve stops on it.  Costs one vector of Z per
// step beside V.
static cs_status gmres_right(const cs_hierarchy *h, cs_cascade *c, const cs_solve_opts *o, const double *b,
                             double *x, double nb, cs_solve_info *inf, cudaStream_t s) {
    const Level &L = h->lev[0];
    const int64_t N = L.g.N;
    const int m = o->restart;
    const bool lowp = o->cycle.precision == CS_FP32, bf16 = o->cycle.precision == CS_BF16;
    if (c->gm_restart < m || !c->gm_Z) {
        dfree(c->gm_V, s); dfree(c->gm_h, s); dfree(c->gm_Z, s);
        c->gm_V = nullptr; c->gm_h = nullptr; c->gm_Z = nullptr;
        CSX_TRY(dalloc_t(&c->gm_V, (size_t)(m + 1) * N, &c->bytes, s));
        CSX_TRY(dalloc_t(&c->gm_Z, (size_t)m * N, &c->bytes, s));
        CSX_TRY(dalloc_t(&c->gm_h, (size_t)(m + 2) * 2, &c->bytes, s));
        c->gm_restart = m;
    }
    double *V = c->gm_V, *Z = c->gm_Z, *hd = c->gm_h;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m), hh(m + 2);
    // Z_j = M v: the cycle output of the right-hand side v, in FP64
    auto precond_to = [&](const double *v, double *zout) -> cs_status {
        if (lowp) {
            CSX_TRY(launch_copy_d2f(N, v, c->lo[0].b, s));
            CSX_TRY(run_v0(h, c, o->cycle, s));
            CSX_CUDA(cudaMemsetAsync(zout, 0, sizeof(double) * N, s));
            CSX_TRY(launch_axpy_f32(N, c->lo[0].x, zout, s));
        } else if (bf16) {
            CSX_TRY(launch_copy_d2bf(N, v, c->lo16[0].b, s));
            CSX_TRY(run_v0(h, c, o->cycle, s));
            CSX_CUDA(cudaMemsetAsync(zout, 0, sizeof(double) * N, s));
            CSX_TRY(launch_axpy_bf16(N, c->lo16[0].x, zout, s));
        } else {
            CSX_CUDA(cudaMemcpyAsync(L.b, v, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
            CSX_TRY(run_v0(h, c, o->cycle, s));
            CSX_CUDA(cudaMemcpyAsync(zout, L.x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        }
        return CS_OK;
    };
    auto dot_to = [&](const double *a, const double *bb, double *dst) -> cs_status {
        CSX_TRY(launch_dot(N, a, bb, h->red, NRED, s));
        CSX_CUDA(cudaMemcpyAsync(dst, h->red + NRED, sizeof(double), cudaMemcpyDeviceToDevice, s));
        return CS_OK;
    };
    const int nred = residual_blocks(L);
    double rel = 1.0;
    cs_status rc = CS_OK;
    for (;;) {
        CSX_TRY(launch_residual64(L, L.A, b, x, L.t, nullptr, h->red, nred, s));  // L.t = b - A x
        rel = std::sqrt(host_sum(h, nred, s, &rc)) / nb;
        if (rc != CS_OK) return rc;
        if (!std::isfinite(rel)) { set_error("GMRES diverged"); return CS_ERR_DIVERGED; }
        if (inf->nhist == 0 && o->hist && inf->nhist < o->hist_cap) o->hist[inf->nhist++] = rel;
        if (rel <= o->tol || inf->iterations >= o->maxit) break;
        CSX_TRY(dot_to(L.t, L.t, hd));
        CSX_TRY(launch_scale_dev(N, hd, V, L.t, s));
        CSX_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double), cudaMemcpyDeviceToHost, s));
        CSX_CUDA(cudaStreamSynchronize(s));
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = std::sqrt(hh[0]);
        int j;
        for (j = 0; j < m && inf->iterations < o->maxit; ++j) {
            double *zj = Z + (int64_t)j * N, *w = V + (int64_t)(j + 1) * N;
            CSX_TRY(precond_to(V + (int64_t)j * N, zj));
            ++inf->iterations;
            CSX_TRY(launch_matvec64(L, L.A, zj, w, s));
            for (int i = 0; i <= j; ++i) {
                CSX_TRY(dot_to(w, V + (int64_t)i * N, hd + i));
                CSX_TRY(launch_axpy_dev(N, hd + i, -1.0, V + (int64_t)i * N, w, s));
            }
            CSX_TRY(dot_to(w, w, hd + j + 1));
            CSX_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
            CSX_CUDA(cudaStreamSynchronize(s));
            double hn = std::sqrt(hh[j + 1]);
            if (hn > 0.0) CSX_TRY(launch_scale_dev(N, hd + j + 1, w, w, s));
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i];
            H[(size_t)(j + 1) * m + j] = hn;
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * bb;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
            double d = std::sqrt(a * a + bb * bb);
            cs[j] = d > 0 ? a / d : 1.0;
            sn[j] = d > 0 ? bb / d : 0.0;
            H[(size_t)j * m + j] = d;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (o->hist && inf->nhist < o->hist_cap) o->hist[inf->nhist++] = std::fabs(g[j + 1]) / nb;
            if (std::fabs(g[j + 1]) <= o->tol * nb || hn == 0.0) { ++j; break; }
        }
        for (int i = j - 1; i >= 0; --i) {
            double sum = g[i];
            for (int k = i + 1; k < j; ++k) sum -= H[(size_t)i * m + k] * y[k];
            y[i] = sum / H[(size_t)i * m + i];
        }
        CSX_CUDA(cudaMemcpyAsync(hd, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
        CSX_TRY(launch_axpy_multi(N, j, hd, Z, x, s));
        CSX_CUDA(cudaStreamSynchronize(s));  // y is a host buffer reused next restart
    }
    inf->final_rel_residual = rel;
    inf->converged = rel <= o->tol;
    if (!inf->converged) {
        set_error("GMRES not converged after %d iterations (relative residual %g)", inf->iterations, rel);
        return CS_ERR_NOTCONV;
    }
    return CS_OK;
}

cs_status cs_query_level(const cs_hierarchy *h, int level, cs_level_info *info) {
    if (!h || !info) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    const Level &L = h->lev[level];
    info->dim = L.g.dim;
    info->n[0] = L.g.nx; info->n[1] = L.g.ny; info->n[2] = L.g.nz;
    info->N = L.g.N;
    info->nst = L.nst;
    for (int s = 0; s < 27; ++s)
        for (int d = 0; d < 3; ++d) info->off[s][d] = s < L.nst ? L.off[s][d] : 0;
    info->nlevels = h->nlev;
    info->block = L.bs;
    int64_t ls = 0;
    if (L.bs == 1) ls = L.g.N;
    else
        for (int64_t b = 0; b < L.nblocks; ++b) {
            const int bx = (int)(b % L.nbx), by = (int)((b / L.nbx) % L.nby), bz = (int)(b / ((int64_t)L.nbx * L.nby));
            const int64_t ex = std::min(L.bs, L.g.nx - L.bs * bx), ey = std::min(L.bs, L.g.ny - L.bs * by);
            const int64_t ez = L.g.dim == 3 ? std::min(L.bs, L.g.nz - L.bs * bz) : 1;
            ls += (ex * ey * ez) * (ex * ey * ez);
        }
    info->lamsize = ls;
    info->sym32 = L.sym32;
    return CS_OK;
}

cs_status cs_export_operator(const cs_hierarchy *h, int level, double *host) {
    if (!h || !host) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    const Level &L = h->lev[level];
    CSX_CUDA(cudaDeviceSynchronize());
    CSX_CUDA(cudaMemcpy(host, L.A, sizeof(double) * L.nst * L.g.N, cudaMemcpyDeviceToHost));
    return CS_OK;
}

cs_status cs_export_colours(const cs_hierarchy *h, int level, int8_t *host) {
    if (!h || !host) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= h->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    const Grid &g = h->lev[level].g;
    for (int iz = 0; iz < g.nz; ++iz)
        for (int iy = 0; iy < g.ny; ++iy)
            for (int ix = 0; ix < g.nx; ++ix)
                host[ix + (int64_t)g.nx * (iy + (int64_t)g.ny * iz)] =
                    (int8_t)(((ix + 1) + (iy + 1) + (g.dim == 3 ? iz + 1 : 0)) & 1);
    return CS_OK;
}

cs_status cs_export_lambda(const cs_cascade *c, int level, double *host) {
    if (!c || !host) { set_error("null argument"); return CS_ERR_ARG; }
    if (level < 0 || level >= c->nlev) { set_error("bad level"); return CS_ERR_ARG; }
    CSX_CUDA(cudaDeviceSynchronize());
    const Level &L = c->h->lev[level];
    if (L.bs == 1) {
        CSX_CUDA(cudaMemcpy(host, c->lam[level], sizeof(double) * c->nu * L.g.N, cudaMemcpyDeviceToHost));
        return CS_OK;
    }
    // blocks: n_b x n_b per block over its nodes in ascending index order
    const int64_t stride = lam_step(L);
    std::vector<double> full((size_t)c->nu * stride);
    CSX_CUDA(cudaMemcpy(full.data(), c->lam[level], sizeof(double) * full.size(), cudaMemcpyDeviceToHost));
    int64_t k = 0;
    for (int st = 0; st < c->nu; ++st)
        for (int64_t b = 0; b < L.nblocks; ++b) {
            const int bx = (int)(b % L.nbx), by = (int)((b / L.nbx) % L.nby), bz = (int)(b / ((int64_t)L.nbx * L.nby));
            int lp[27], np = 0;
            for (int q = 0; q < L.nmax; ++q) {
                const int lx = q % L.bs, ly = (q / L.bs) % L.bs, lz = L.g.dim == 3 ? q / (L.bs * L.bs) : 0;
                if (L.bs * bx + lx < L.g.nx && L.bs * by + ly < L.g.ny && (L.g.dim == 2 || L.bs * bz + lz < L.g.nz))
                    lp[np++] = q;
            }
            const double *src = full.data() + st * stride + b * L.nmax * L.nmax;
            for (int p = 0; p < np; ++p)
                for (int q = 0; q < np; ++q) host[k++] = src[lp[p] * L.nmax + lp[q]];
        }
    return CS_OK;
}

}  // extern "C"
