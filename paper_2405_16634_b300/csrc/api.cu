// api.cu -- the extern "C" boundary (include/wnnc.h): argument checks, status
// codes, thread-local error text, tree lifetime and work buffers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>

#include "common.cuh"

namespace wnnc {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_last_error(const std::string& msg) { g_last_error = msg; }

[[noreturn]] void fail(wnnc_status st, const std::string& msg) { throw Error{st, msg}; }

// ---------------------------------------------------------------------------
// Stream-ordered memory pool (one per device, created on first use).  Its
// release threshold is unlimited, so memory freed back to it stays reserved
// for the next allocation instead of returning to the driver.
// ---------------------------------------------------------------------------
cudaStream_t& alloc_stream() {
    static thread_local cudaStream_t s = nullptr;
    return s;
}

namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaMemPool_t pool_for_current_device() {
    int dev = 0;
    WNNC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxPoolDevices) fail(WNNC_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        WNNC_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t keep = UINT64_MAX;
        WNNC_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pools[dev] = p;
    }
    return g_pools[dev];
}
}  // namespace

// Fault injection on the host (wnnc_debug_fail_alloc): device allocations
// left before the next one fails with WNNC_ENOMEM; -1 = off.
static std::atomic<int64_t> g_fail_alloc_after{-1};

void* pool_alloc(size_t bytes) {
    int64_t k = g_fail_alloc_after.load();
    while (k >= 0 && !g_fail_alloc_after.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) fail(WNNC_ENOMEM, "injected device allocation failure (wnnc_debug_fail_alloc)");
    void* p = nullptr;
    WNNC_CUDA(cudaMallocFromPoolAsync(&p, bytes, pool_for_current_device(), alloc_stream()));
    return p;
}

void pool_free(void* p) {
    if (p) cudaFreeAsync(p, alloc_stream());
}

static void alloc_workspace(Tree& t) {
    const int64_t n = t.n;
    const int nn = t.nnodes;
    t.mu_a = dalloc<float4>(n);
    t.mu_b = dalloc<float4>(n);
    t.r_s = dalloc<float4>(n);
    t.g_mu = dalloc<float4>(n);
    t.g_r = dalloc<float4>(n);
    t.s_s = dalloc<float>(n);
    t.area_s = dalloc<float>(n);
    t.mom = dalloc<float4>(nn);
    t.mom_r = dalloc<float4>(nn);
    t.node_rep = dalloc<float4>(nn);
    t.contrib = dalloc<float4>(t.self.far_entries);
    t.near_contrib = dalloc<float4>(t.near_slots);
    t.vnode = dalloc<float4>(nn);
    t.mom_x = dalloc<float4>(nn);
    if (t.params.moments_fp64) t.dmom = dalloc<double>(8 * (size_t)nn);
    t.partials = dalloc<double>(3 * (size_t)std::max(std::max(t.self.ngroups, t.self.nchunks), t.nach));
    t.red = dalloc<double>(3 * 256);
    t.red_ticket = dalloc<unsigned>(1);
    WNNC_CUDA(cudaMemsetAsync(t.red_ticket, 0, sizeof(unsigned), alloc_stream()));
    t.part_slots = std::max(t.self.work.nslots, t.adj_near_work.nslots);
    t.part_acc = dalloc<float4>((size_t)t.part_slots * 32);
    t.scalars = dalloc<double>(4);
    WNNC_CUDA(cudaMemsetAsync(t.scalars, 0, 4 * sizeof(double), alloc_stream()));
    t.err_flag = dalloc<int>(1);
    WNNC_CUDA(cudaMemsetAsync(t.err_flag, 0, sizeof(int), alloc_stream()));
    if (!t.aux) WNNC_CUDA(cudaStreamCreateWithFlags(&t.aux, cudaStreamNonBlocking));
    WNNC_CUDA(cudaEventCreateWithFlags(&t.ev_fork, cudaEventDisableTiming));
    WNNC_CUDA(cudaEventCreateWithFlags(&t.ev_join, cudaEventDisableTiming));
    if (t.params.far_order == 1) {
        t.mom_dip = dalloc<float4>(2 * (size_t)nn);
        t.mom_dip_r = dalloc<float4>(2 * (size_t)nn);
        t.dip_corr = dalloc<float4>(n);
        t.contrib_h0 = dalloc<float4>(t.self.far_entries);
        t.contrib_h1 = dalloc<float4>(t.self.far_entries);
        t.hnode0 = dalloc<float4>(nn);
        t.hnode1 = dalloc<float4>(nn);
    }
    if (t.self.far_lsplit) {
        t.dip_corr = dalloc<float4>(n);   // per-target terms of the expanded entries
        t.gather_raw = dalloc<float4>(n);
        t.node_abs = dalloc<float4>(nn);
        t.local_rec = dalloc<float4>(2 * (size_t)nn);
        t.gadj = dalloc<float4>(2 * (size_t)t.self.ngroups);
        if (t.self.nclusters) t.cadj = dalloc<float4>(2 * (size_t)t.self.nclusters);
        local_setup(t, alloc_stream());
    }
}

// Read and clear the latched device error flags.
static wnnc_status take_device_status(Tree& t, cudaStream_t s) {
    int f = 0;
    WNNC_CUDA(cudaMemcpyAsync(&f, t.err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    WNNC_CUDA(cudaStreamSynchronize(s));
    if (f) {
        WNNC_CUDA(cudaMemsetAsync(t.err_flag, 0, sizeof(int), s));
        WNNC_CUDA(cudaStreamSynchronize(s));
        if (f & kErrNonFinite) {
            set_last_error("non-finite step length in the iteration");
            return WNNC_ENONFINITE;
        }
        set_last_error("device capacity exceeded");
        return WNNC_ECAPACITY;
    }
    return WNNC_OK;
}

template <class F>
static wnnc_status guarded(F&& f) {
    try {
        f();
        return WNNC_OK;
    } catch (const Error& e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc&) {
        set_last_error("host allocation failed");
        return WNNC_ENOMEM;
    } catch (...) {
        set_last_error("unexpected internal error");
        return WNNC_ECUDA;
    }
}

static void check_params(const wnnc_tree_params& p) {
    if (p.max_depth < 1 || p.max_depth > kMaxDepth) fail(WNNC_EINVAL, "max_depth must be in [1, 15]");
    if (p.leaf_size < 1 || p.leaf_size > 1024) fail(WNNC_EINVAL, "leaf_size must be in [1, 1024]");
    if (!(p.theta >= 0.f) || !std::isfinite(p.theta)) fail(WNNC_EINVAL, "theta must be finite and >= 0");
    if (p.rep_mode != 0 && p.rep_mode != 1) fail(WNNC_EINVAL, "rep_mode must be 0 or 1");
    if (p.near_bf16 != 0 && p.near_bf16 != 1) fail(WNNC_EINVAL, "near_bf16 must be 0 or 1");
    if (p.criterion != 0 && p.criterion != 1) fail(WNNC_EINVAL, "criterion must be 0 or 1");
    if (p.criterion == 1 && (p.rep_mode != 0 || p.near_bf16 != 0))
        fail(WNNC_EINVAL, "criterion 1 (per-target Alg. 4) needs rep_mode 0 and near_bf16 0");
    if (p.far_order != 0 && p.far_order != 1) fail(WNNC_EINVAL, "far_order must be 0 or 1");
    if (p.far_order == 1 && (p.rep_mode != 1 || p.criterion != 0))
        fail(WNNC_EINVAL, "far_order 1 needs rep_mode 1 and criterion 0");
    if (!(p.local_theta >= 0.f) || !std::isfinite(p.local_theta))
        fail(WNNC_EINVAL, "local_theta must be finite and >= 0");
    if (p.local_theta > 0.f && (p.rep_mode != 1 || p.criterion != 0 || p.far_order != 0))
        fail(WNNC_EINVAL, "local_theta > 0 needs rep_mode 1, criterion 0 and far_order 0");
    if (p.local_cluster != 0 && (p.local_cluster < 2 || p.local_cluster > kMaxCluster))
        fail(WNNC_EINVAL, "local_cluster must be 0 or in [2, 8]");
    if (p.local_cluster != 0 && !(p.local_theta > 0.f))
        fail(WNNC_EINVAL, "local_cluster needs local_theta > 0");
}

static void check_w(float w) {
    if (!(w >= 0.f) || !std::isfinite(w)) fail(WNNC_EINVAL, "w must be finite and >= 0");
}

static Tree& unwrap(const wnnc_tree* h) {
    if (!h) fail(WNNC_EINVAL, "tree is NULL");
    return *reinterpret_cast<Tree*>(const_cast<wnnc_tree*>(h));
}

}  // namespace wnnc

using namespace wnnc;

extern "C" {

wnnc_status wnnc_tree_params_default(wnnc_tree_params* p) {
    if (!p) {
        set_last_error("params is NULL");
        return WNNC_EINVAL;
    }
    p->max_depth = 15;
    p->leaf_size = 8;
    p->theta = 0.5f;
    p->rep_mode = 1;
    p->moments_fp64 = 0;
    p->near_bf16 = 0;
    p->criterion = 0;
    p->far_order = 0;
    p->local_theta = 0.f;
    p->local_cluster = 0;
    return WNNC_OK;
}

wnnc_status wnnc_iter_params_default(wnnc_iter_params* p) {
    if (!p) {
        set_last_error("params is NULL");
        return WNNC_EINVAL;
    }
    p->n_iter = 40;
    p->first_iter = 1;
    p->last_iter = 0;
    p->w1 = 0.002f;
    p->w2 = 0.016f;
    p->init = 0;
    p->rescale = 0;
    p->use_grad = 1;
    p->use_wnnc = 1;
    p->schedule = 0;
    return WNNC_OK;
}

wnnc_status wnnc_debug_fail_alloc(int64_t after) {
    g_fail_alloc_after.store(after < 0 ? -1 : after);
    return WNNC_OK;
}

// A stream of the highest priority for one build, ordered after the caller's
// stream at creation (fork) and before it again at join().
struct BuildStream {
    cudaStream_t us, s = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    explicit BuildStream(cudaStream_t caller) : us(caller) {
        int least = 0, greatest = 0;
        WNNC_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        WNNC_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest));
        WNNC_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        WNNC_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        WNNC_CUDA(cudaEventRecord(fork, us));
        WNNC_CUDA(cudaStreamWaitEvent(s, fork, 0));
    }
    void join() {
        WNNC_CUDA(cudaEventRecord(done, s));
        WNNC_CUDA(cudaStreamWaitEvent(us, done, 0));
    }
    ~BuildStream() {
        if (done) cudaEventDestroy(done);
        if (fork) cudaEventDestroy(fork);
        if (s) cudaStreamDestroy(s);
    }
    BuildStream(const BuildStream&) = delete;
    BuildStream& operator=(const BuildStream&) = delete;
};

wnnc_status wnnc_build_tree(const float* pts, int64_t n, const wnnc_tree_params* params, void* stream,
                            wnnc_tree** out) {
    if (out) *out = nullptr;
    Tree* t = nullptr;
    wnnc_status st = guarded([&] {
        if (!out) fail(WNNC_EINVAL, "out is NULL");
        if (!pts) fail(WNNC_EINVAL, "pts is NULL");
        if (n < 1) fail(WNNC_EINVAL, "n must be >= 1");
        if (n > (int64_t)INT32_MAX / 2) fail(WNNC_EINVAL, "n too large (max 2^30 points)");
        wnnc_tree_params p;
        wnnc_tree_params_default(&p);
        if (params) p = *params;
        check_params(p);
        t = new Tree();
        t->n = n;
        t->params = p;
        WNNC_CUDA(cudaGetDevice(&t->device));
        cudaStream_t us = static_cast<cudaStream_t>(stream);
        // the build runs on a stream of the highest priority, after the work
        // queued on the caller's stream and before what follows there: its
        // short kernels then go ahead of the transposed lists' sorts on the
        // second stream
        BuildStream bs(us);
        cudaStream_t s = bs.s;
        {
            AllocStream as(s);
            build_tree(*t, pts, s);
            alloc_workspace(*t);
        }
        bs.join();
        unsigned timeouts = 0;
        wait_timeouts_async(&timeouts, us);
        WNNC_CUDA(cudaStreamSynchronize(us));
        check_wait_timeouts(timeouts, us);
    });
    if (st != WNNC_OK) {
        if (t) {
            cudaDeviceSynchronize();
            free_tree(*t);
            delete t;
        }
        return st;
    }
    *out = reinterpret_cast<wnnc_tree*>(t);
    return WNNC_OK;
}

wnnc_status wnnc_tree_free(wnnc_tree* tree) {
    if (!tree) return WNNC_OK;
    return guarded([&] {
        Tree* t = reinterpret_cast<Tree*>(tree);
        WNNC_CUDA(cudaDeviceSynchronize());
        free_tree(*t);
        delete t;
    });
}

wnnc_status wnnc_eval_w(const wnnc_tree* tree, const float* mu, float w, float* out, void* stream) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (!mu || !out) fail(WNNC_EINVAL, "mu/out is NULL");
        check_w(w);
        eval_w(t, mu, w, out, static_cast<cudaStream_t>(stream));
    });
}

wnnc_status wnnc_eval_grad(const wnnc_tree* tree, const float* mu, float w, float* out, void* stream) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (!mu || !out) fail(WNNC_EINVAL, "mu/out is NULL");
        check_w(w);
        eval_grad(t, mu, w, out, static_cast<cudaStream_t>(stream));
    });
}

wnnc_status wnnc_eval_adjoint(const wnnc_tree* tree, const float* s, float w, float* out, void* stream) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (!s || !out) fail(WNNC_EINVAL, "s/out is NULL");
        check_w(w);
        eval_adjoint(t, s, w, out, static_cast<cudaStream_t>(stream));
    });
}

wnnc_status wnnc_eval_at(const wnnc_tree* tree, const float* mu, const float* q, int64_t m, float w,
                         int grad, float* out, void* stream) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (!mu || !q || !out) fail(WNNC_EINVAL, "mu/q/out is NULL");
        if (m < 1) fail(WNNC_EINVAL, "m must be >= 1");
        if (m > (int64_t)INT32_MAX / 2) fail(WNNC_EINVAL, "m too large");
        check_w(w);
        AllocStream as(static_cast<cudaStream_t>(stream));
        eval_at(t, mu, q, m, w, grad, out, static_cast<cudaStream_t>(stream));
    });
}

wnnc_status wnnc_iterate(wnnc_tree* tree, float* mu_inout, const float* area, const wnnc_iter_params* params,
                         void* stream, float* stats) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (!mu_inout) fail(WNNC_EINVAL, "mu_inout is NULL");
        wnnc_iter_params p;
        wnnc_iter_params_default(&p);
        if (params) p = *params;
        const int last = p.last_iter > 0 ? p.last_iter : p.n_iter;
        if (p.n_iter < 1) fail(WNNC_EINVAL, "n_iter must be >= 1");
        if (p.first_iter < 1 || p.first_iter > last || last > p.n_iter)
            fail(WNNC_EINVAL, "need 1 <= first_iter <= last_iter <= n_iter");
        check_w(p.w1);
        check_w(p.w2);
        if (p.init != 0 && p.init != 1) fail(WNNC_EINVAL, "init must be 0 or 1");
        if (p.rescale != 0 && p.rescale != 1) fail(WNNC_EINVAL, "rescale must be 0 or 1");
        if (p.rescale == 1 && !area) fail(WNNC_EINVAL, "rescale = 1 needs area");
        if (p.schedule < 0 || p.schedule > 2) fail(WNNC_EINVAL, "schedule must be 0, 1 or 2");
        if (p.schedule == 2 && !(p.w1 > 0.f && p.w2 > 0.f))
            fail(WNNC_EINVAL, "the exponential schedule needs w1 > 0 and w2 > 0");
        iterate(t, mu_inout, area, p, static_cast<cudaStream_t>(stream), stats);
    });
}

wnnc_status wnnc_orient(const float* pts_host, int64_t n, const wnnc_tree_params* tree_params,
                        const wnnc_iter_params* iter_params, const float* area_host, float* mu_host,
                        void* stream) {
    float* dpts = nullptr;
    float* dmu = nullptr;
    float* darea = nullptr;
    wnnc_tree* tree = nullptr;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    wnnc_status st = guarded([&] {
        if (!pts_host || !mu_host) fail(WNNC_EINVAL, "pts_host/mu_host is NULL");
        if (n < 1) fail(WNNC_EINVAL, "n must be >= 1");
        if (n > (int64_t)INT32_MAX / 2) fail(WNNC_EINVAL, "n too large (max 2^30 points)");
        wnnc_iter_params p;
        wnnc_iter_params_default(&p);
        if (iter_params) p = *iter_params;
        if (p.rescale == 1 && !area_host) fail(WNNC_EINVAL, "rescale = 1 needs area_host");
        AllocStream as(s);
        const size_t bytes = sizeof(float) * 3 * (size_t)n;
        dpts = dalloc<float>(3 * (size_t)n);
        dmu = dalloc<float>(3 * (size_t)n);
        WNNC_CUDA(cudaMemcpyAsync(dpts, pts_host, bytes, cudaMemcpyHostToDevice, s));
        if (p.init == 1) WNNC_CUDA(cudaMemcpyAsync(dmu, mu_host, bytes, cudaMemcpyHostToDevice, s));
        if (area_host) {
            darea = dalloc<float>((size_t)n);
            WNNC_CUDA(cudaMemcpyAsync(darea, area_host, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, s));
        }
        wnnc_status b = wnnc_build_tree(dpts, n, tree_params, stream, &tree);
        if (b != WNNC_OK) fail(b, wnnc_last_error());
        b = wnnc_iterate(tree, dmu, darea, &p, stream, nullptr);
        if (b != WNNC_OK) fail(b, wnnc_last_error());
        WNNC_CUDA(cudaMemcpyAsync(mu_host, dmu, bytes, cudaMemcpyDeviceToHost, s));
        WNNC_CUDA(cudaStreamSynchronize(s));
        b = wnnc_sync_status(tree, stream);
        if (b != WNNC_OK) fail(b, wnnc_last_error());
    });
    if (st != WNNC_OK) cudaStreamSynchronize(s);
    if (tree) wnnc_tree_free(tree);
    {
        AllocStream as(s);
        pool_free(dpts);
        pool_free(dmu);
        pool_free(darea);
    }
    return st;
}

wnnc_status wnnc_get_stats(const wnnc_tree* tree, int64_t* far_pairs, int64_t* near_pairs) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (far_pairs) *far_pairs = t.self.far_pairs;
        if (near_pairs) *near_pairs = t.self.near_pairs;
    });
}

wnnc_status wnnc_get_local_stats(const wnnc_tree* tree, int64_t* local_entries, int64_t* local_pairs) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (local_entries) *local_entries = t.self.local_entries;
        if (local_pairs) *local_pairs = t.self.local_pairs;
    });
}

wnnc_status wnnc_get_cluster_stats(const wnnc_tree* tree, int64_t* cluster_entries, int64_t* cluster_pairs) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (cluster_entries) *cluster_entries = t.self.cluster_entries;
        if (cluster_pairs) *cluster_pairs = t.self.cluster_pairs;
    });
}

wnnc_status wnnc_tree_info(const wnnc_tree* tree, int64_t* n, int64_t* nnodes, int64_t* nleaves,
                           int64_t* ngroups, int64_t* far_entries, int64_t* near_ranges,
                           int64_t* tnear_entries, int* depth) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (n) *n = t.n;
        if (nnodes) *nnodes = t.nnodes;
        if (nleaves) *nleaves = t.nleaves;
        if (ngroups) *ngroups = t.self.ngroups;
        if (far_entries) *far_entries = t.self.far_entries;
        if (near_ranges) *near_ranges = t.self.near_ranges;
        if (tnear_entries) *tnear_entries = t.tnear_entries;
        if (depth) *depth = t.depth_reached;
    });
}

wnnc_status wnnc_tree_walk_stats(const wnnc_tree* tree, int* stack_walk_groups, int* big_stack) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (stack_walk_groups) *stack_walk_groups = t.self.walk_stack_groups;
        if (big_stack) *big_stack = t.self.walk_big_stack;
    });
}

wnnc_status wnnc_tree_export(const wnnc_tree* tree, int64_t* perm, int32_t* node_start, int32_t* node_count,
                             int32_t* node_depth, int32_t* node_nchild, int32_t* far_off, int32_t* far_id,
                             int32_t* near_off, int32_t* near_rng, int32_t* group_off,
                             double* center_scale) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        WNNC_CUDA(cudaDeviceSynchronize());
        auto cp = [](void* dst, const void* src, size_t bytes) {
            if (dst && bytes) WNNC_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
        };
        const TargetSet& S = t.self;
        cp(perm, S.perm, sizeof(int64_t) * t.n);
        cp(node_start, t.node_start, sizeof(int) * t.nnodes);
        cp(node_count, t.node_count, sizeof(int) * t.nnodes);
        cp(node_depth, t.node_depth, sizeof(int) * t.nnodes);
        cp(node_nchild, t.node_nchild, sizeof(int) * t.nnodes);
        cp(far_off, S.far_off, sizeof(int) * (S.ngroups + 1));
        cp(far_id, S.far_id, sizeof(int) * S.far_entries);
        cp(near_off, S.near_off, sizeof(int) * (S.ngroups + 1));
        cp(near_rng, S.near_rng, sizeof(int2) * S.near_ranges);
        cp(group_off, S.goff, sizeof(int) * (S.ngroups + 1));
        if (center_scale) {
            for (int k = 0; k < 3; ++k) center_scale[k] = t.center[k];
            center_scale[3] = t.scale;
        }
    });
}

wnnc_status wnnc_tree_export_local(const wnnc_tree* tree, int32_t* far_lsplit, int32_t* far_csplit) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        if (!far_lsplit || !far_csplit) fail(WNNC_EINVAL, "far_lsplit or far_csplit is NULL");
        WNNC_CUDA(cudaDeviceSynchronize());
        const TargetSet& S = t.self;
        if (S.ngroups == 0) return;
        const int* ls = S.far_lsplit ? S.far_lsplit : S.far_off + 1;
        const int* cs = S.far_csplit ? S.far_csplit : S.far_off + 1;
        WNNC_CUDA(cudaMemcpy(far_lsplit, ls, sizeof(int) * S.ngroups, cudaMemcpyDeviceToHost));
        WNNC_CUDA(cudaMemcpy(far_csplit, cs, sizeof(int) * S.ngroups, cudaMemcpyDeviceToHost));
    });
}

wnnc_status wnnc_profile_enable(wnnc_tree* tree, int enable) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        t.prof.on = enable != 0;
    });
}

wnnc_status wnnc_profile_classes(wnnc_tree* tree, unsigned mask) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        t.prof.mask = mask;
    });
}

wnnc_status wnnc_profile_read(wnnc_tree* tree, int64_t* launches, double* total_ms) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        t.prof.collect();
        for (int k = 0; k < WNNC_PROF_CLASSES; ++k) {
            if (launches) launches[k] = t.prof.launches[k];
            if (total_ms) total_ms[k] = t.prof.ms[k];
        }
    });
}

wnnc_status wnnc_profile_reset(wnnc_tree* tree) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        t.prof.reset();
    });
}

wnnc_status wnnc_sync_status(wnnc_tree* tree, void* stream) {
    wnnc_status dev = WNNC_OK;
    wnnc_status st = guarded([&] {
        Tree& t = unwrap(tree);
        dev = take_device_status(t, static_cast<cudaStream_t>(stream));
    });
    return st != WNNC_OK ? st : dev;
}

wnnc_status wnnc_knn16(const wnnc_tree* tree, int32_t* idx, float* feat, void* stream) {
    return guarded([&] {
        Tree& t = unwrap(tree);
        AllocStream as(static_cast<cudaStream_t>(stream));
        knn16(t, idx, feat, static_cast<cudaStream_t>(stream));
    });
}

static Mlp& unwrap_mlp(const wnnc_mlp* h) {
    if (!h) fail(WNNC_EINVAL, "mlp is NULL");
    return *reinterpret_cast<Mlp*>(const_cast<wnnc_mlp*>(h));
}

wnnc_status wnnc_mlp_create(int64_t max_batch, wnnc_mlp** out) {
    if (out) *out = nullptr;
    Mlp* m = nullptr;
    wnnc_status st = guarded([&] {
        if (!out) fail(WNNC_EINVAL, "out is NULL");
        if (max_batch < 1 || max_batch > (int64_t)1 << 26) fail(WNNC_EINVAL, "max_batch must be in [1, 2^26]");
        m = new Mlp();
        mlp_alloc(*m, max_batch);
        WNNC_CUDA(cudaStreamSynchronize(alloc_stream()));   // allocations complete before any stream uses them
    });
    if (st != WNNC_OK) {
        if (m) {
            mlp_free(*m);
            delete m;
        }
        return st;
    }
    *out = reinterpret_cast<wnnc_mlp*>(m);
    return WNNC_OK;
}

wnnc_status wnnc_mlp_free(wnnc_mlp* mlp) {
    if (!mlp) return WNNC_OK;
    return guarded([&] {
        Mlp* m = reinterpret_cast<Mlp*>(mlp);
        WNNC_CUDA(cudaDeviceSynchronize());
        mlp_free(*m);
        delete m;
    });
}

wnnc_status wnnc_mlp_set_params(wnnc_mlp* mlp, const float* params, void* stream) {
    return guarded([&] {
        Mlp& m = unwrap_mlp(mlp);
        if (!params) fail(WNNC_EINVAL, "params is NULL");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t bytes = sizeof(float) * mlp_param_count();
        WNNC_CUDA(cudaMemcpyAsync(m.params, params, bytes, cudaMemcpyDeviceToDevice, s));
        WNNC_CUDA(cudaMemsetAsync(m.m, 0, bytes, s));
        WNNC_CUDA(cudaMemsetAsync(m.v, 0, bytes, s));
        m.step = 0;
    });
}

wnnc_status wnnc_mlp_get_params(const wnnc_mlp* mlp, float* params, void* stream) {
    return guarded([&] {
        Mlp& m = unwrap_mlp(mlp);
        if (!params) fail(WNNC_EINVAL, "params is NULL");
        WNNC_CUDA(cudaMemcpyAsync(params, m.params, sizeof(float) * mlp_param_count(), cudaMemcpyDeviceToDevice,
                                  static_cast<cudaStream_t>(stream)));
    });
}

wnnc_status wnnc_mlp_forward(wnnc_mlp* mlp, const float* x, int64_t B, float* y, void* stream) {
    return guarded([&] {
        Mlp& m = unwrap_mlp(mlp);
        if (!x || !y) fail(WNNC_EINVAL, "x/y is NULL");
        if (B < 1) fail(WNNC_EINVAL, "B must be >= 1");
        mlp_forward(m, x, B, y, static_cast<cudaStream_t>(stream));
    });
}

wnnc_status wnnc_mlp_set_loss(wnnc_mlp* mlp, int mode) {
    return guarded([&] {
        Mlp& m = unwrap_mlp(mlp);
        if (mode != 0 && mode != 1) fail(WNNC_EINVAL, "loss mode must be 0 or 1");
        m.loss_mode = mode;
    });
}

wnnc_status wnnc_mlp_grad(wnnc_mlp* mlp, const float* x, const float* label, int64_t B, float* grad, float* loss,
                          void* stream) {
    return guarded([&] {
        Mlp& m = unwrap_mlp(mlp);
        if (!x || !label) fail(WNNC_EINVAL, "x/label is NULL");
        if (B < 1 || B > m.max_batch) fail(WNNC_EINVAL, "B must be in [1, max_batch]");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        mlp_grad(m, x, label, B, loss, s);
        if (grad)
            WNNC_CUDA(cudaMemcpyAsync(grad, m.grad, sizeof(float) * mlp_param_count(), cudaMemcpyDeviceToDevice, s));
    });
}

wnnc_status wnnc_mlp_train_step(wnnc_mlp* mlp, const float* x, const float* label, int64_t B, float lr, float* loss,
                                void* stream) {
    return guarded([&] {
        Mlp& m = unwrap_mlp(mlp);
        if (!x || !label) fail(WNNC_EINVAL, "x/label is NULL");
        if (B < 1 || B > m.max_batch) fail(WNNC_EINVAL, "B must be in [1, max_batch]");
        if (!(lr > 0.f) || !std::isfinite(lr)) fail(WNNC_EINVAL, "lr must be finite and > 0");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        mlp_grad(m, x, label, B, loss, s);
        mlp_adam(m, lr, s);
    });
}

wnnc_status wnnc_warm_init(const float* dir, const float* ref, int64_t n, float area, float* mu, void* stream) {
    return guarded([&] {
        if (!dir || !mu) fail(WNNC_EINVAL, "dir/mu is NULL");
        if (n < 1) fail(WNNC_EINVAL, "n must be >= 1");
        if (!(area >= 0.f) || !std::isfinite(area)) fail(WNNC_EINVAL, "area must be finite and >= 0");
        warm_init(dir, ref, n, area, mu, static_cast<cudaStream_t>(stream));
    });
}

int64_t wnnc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

wnnc_status wnnc_probe_fp32(double* tflops, void* stream) {
    return guarded([&] {
        if (!tflops) fail(WNNC_EINVAL, "tflops is NULL");
        AllocStream as(static_cast<cudaStream_t>(stream));
        *tflops = probe_fp32(static_cast<cudaStream_t>(stream));
    });
}

wnnc_status wnnc_selftest_wait_timeout(void* stream) {
    return guarded([&] {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        AllocStream as(s);
        selftest_wait_timeout(s);
    });
}

const char* wnnc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
