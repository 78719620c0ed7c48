// common.cuh -- shared declarations of the WNNC CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/wnnc.h"

namespace wnnc {

constexpr int kWarp = 32;
constexpr int kGroup = 32;          // targets per group = one warp, one target per lane
constexpr int kKeyBits = 45;        // 15 bits per axis -> depth 15
constexpr int kMaxDepth = 15;
constexpr int kMaxCluster = 8;      // largest local_cluster (groups per cluster)
constexpr float kInv4Pi = 0.0795774715459476678f;   // 1/(4 pi)

// Device-side error flags (latched per tree, read by wnnc_sync_status).
enum : int { kErrCapacity = 1, kErrNonFinite = 2 };

// Thrown internally by host orchestration code; converted to a status at the ABI.
struct Error {
    wnnc_status status;
    std::string msg;
};

void set_last_error(const std::string& msg);
[[noreturn]] void fail(wnnc_status st, const std::string& msg);

#define WNNC_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            ::wnnc::fail(e_ == cudaErrorMemoryAllocation ? WNNC_ENOMEM : WNNC_ECUDA,     \
                         std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

// Every kernel launch is followed by this check, which also counts the launch.
void count_launch();
#define WNNC_LAUNCH_CHECK()             \
    do {                                \
        ::wnnc::count_launch();         \
        WNNC_CUDA(cudaGetLastError());  \
    } while (0)

// Device memory comes from the library's own stream-ordered pool on the
// current device, which keeps freed memory for reuse: once it holds enough,
// the temporary buffers of a tree build neither call the driver's allocator
// nor synchronise the device.  Allocations and frees are ordered on the
// stream of the library call in progress on this thread (AllocStream, set by
// the build, query and kNN entry points; the legacy default stream otherwise).
cudaStream_t& alloc_stream();
struct AllocStream {
    cudaStream_t prev;
    explicit AllocStream(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
    ~AllocStream() { alloc_stream() = prev; }
    AllocStream(const AllocStream&) = delete;
    AllocStream& operator=(const AllocStream&) = delete;
};
void* pool_alloc(size_t bytes);     // throws WNNC_ENOMEM / WNNC_ECUDA
void pool_free(void* p);            // no-op for NULL

// Typed device allocation that throws on failure.
template <class T>
T* dalloc(size_t count) {
    if (count == 0) count = 1;
    return static_cast<T*>(pool_alloc(count * sizeof(T)));
}
template <class T>
void dfree(T*& p) {
    pool_free(p);
    p = nullptr;
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Work lists.  A warp processes one Item: a slice of one group's interaction
// lists, at most about `cap` lane-slots long, so that no single warp carries
// a group whose lists are unusually long.  The cap is fixed per list from its
// total cost: about total / kItemsTarget rounded down to a power of two,
// within [kItemCostMin, kItemCostMax], so that small problems still have
// enough items to fill the GPU and large ones keep items long.  Items run
// heaviest first.  When a group is cut into several items, each writes its
// partial sums to a slot of a scratch buffer and a finalize pass adds the
// parts in order.
// ---------------------------------------------------------------------------
#ifndef WNNC_ITEMS_TARGET
#define WNNC_ITEMS_TARGET 8192
#endif
#ifndef WNNC_ITEM_MIN
#define WNNC_ITEM_MIN 256
#endif
constexpr int64_t kItemsTarget = WNNC_ITEMS_TARGET;
constexpr int kItemCostMin = WNNC_ITEM_MIN;    // lane-slots per item (about)
constexpr int kItemCostMax = 4096;
constexpr int kMaxRange = 256;      // near ranges are cut into pieces of at most this many points
constexpr int kAdjChunk = 8;        // points per source chunk of the adjoint near part
constexpr int kMomSmall = 16;       // node moments: nodes of at most this many points, one thread each
constexpr int kMomDirect = 1024;    //   up to this many points, one warp each; larger ones from children
#ifndef WNNC_GROUP_SLACK
#define WNNC_GROUP_SLACK 3
#endif
constexpr int kGroupSlack = WNNC_GROUP_SLACK;      // group rule: see build_target_set
constexpr int kGroupMinDepth = 3;                  // groups stay inside one cell of this depth

struct Item {
    int g;          // target group (adjoint near sums: source chunk)
    int q0, q1;     // near ranges [q0, q1) (adjoint near sums: transposed entries)
    int f0, f1;     // far entries [f0, f1)
    int pslot;      // partial-sum slot if the group is cut into several items, else -1
    int cost;       // lane-slots
    int split;      // the group's record in splits if pslot >= 0, else -1
};

struct WorkList {
    Item* items = nullptr;
    int nitems = 0;
    int4* splits = nullptr;     // (group, first slot, number of parts, -) of cut groups
    unsigned* split_cnt = nullptr;  // per cut group: parts finished (the last one finishes the group)
    int* gsplit = nullptr;      // per group: its record in splits, or -1 (lists with partial sums)
    int nsplit = 0;
    int nslots = 0;
};
void free_work(WorkList& w);

// ---------------------------------------------------------------------------
// Target set: targets sorted by Morton key and cut into groups of at most 32
// consecutive targets (one warp, one target per lane), with the interaction
// lists of each group against the source octree.  Coordinates are stored as
// float offsets from the origin of their fixed 32-point chunk; each group has
// its own origin, and both origins are dyadic so that frame shifts are exact.
// ---------------------------------------------------------------------------
struct TargetSet {
    int64_t m = 0;          // number of targets
    int ngroups = 0;
    int nchunks = 0;
    int64_t* perm = nullptr;      // sorted position -> input index
    float4* pos = nullptr;        // target offset from its chunk origin (x,y,z,0)
    float4* corig = nullptr;      // chunk origins (chunk = 32 consecutive sorted targets)
    float4* gorig = nullptr;      // group origins
    int* goff = nullptr;          // [ngroups+1] group g = sorted targets goff[g]..goff[g+1]-1
    double* glo = nullptr;        // group bounding boxes (3 per group)
    double* ghi = nullptr;
    float4* gbl = nullptr;        // the same boxes in the group's frame, rounded outward
    float4* gbh = nullptr;
    int* far_off = nullptr;       // [ngroups+1]
    int* far_id = nullptr;        // node ids per group: summed pair by pair, then (from
                                  // far_lsplit[g] on) expanded about the group centre;
                                  // ascending within each part
    int* far_lsplit = nullptr;    // [ngroups] first expanded entry of each group (local_theta > 0)
    int* far_csplit = nullptr;    // [ngroups] first entry expanded about the group's cluster
                                  // (local_cluster > 0; the group's expansions end there)
    int nclusters = 0;            // clusters of cluster_k consecutive groups (local_cluster > 0)
    int cluster_k = 0;
    float4* cctr = nullptr;       // [nclusters] cluster frame origin (dyadic) in xyz
    float4* cexp = nullptr;       // [nclusters] expansion centre in that frame and the radius (w)
    float4* gctr = nullptr;       // [ngroups] expansion centre in the group's frame, and the
                                  // group's radius about it (w), rounded up
    int* near_off = nullptr;      // [ngroups+1]
    int2* near_rng = nullptr;     // merged [start,end) source ranges, at most kMaxRange long
    int64_t far_entries = 0, near_ranges = 0;
    int64_t far_pairs = 0, near_pairs = 0;
    int64_t local_entries = 0;    // far entries expanded about the group centre (local_theta > 0)
    int64_t local_pairs = 0;      // the pairs those entries stand for (not in far_pairs)
    int64_t cluster_entries = 0;  // (cluster, node) expansions standing for cluster_pairs of them
    int64_t cluster_pairs = 0;
    // how the list traversal ran: groups that a first-in first-out walk
    // finished as stack walks; whether every group ran again as a stack walk
    // with the larger buffer
    int walk_stack_groups = 0, walk_big_stack = 0;
    WorkList work;                // items of the gather kernels
};

// ---------------------------------------------------------------------------
// Per-launch event timing (wnnc_profile_*).
// ---------------------------------------------------------------------------
struct Profiler {
    bool on = false;
    unsigned mask = ~0u;  // classes recorded while on (bit k: class k)
    struct Rec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    int64_t launches[WNNC_PROF_CLASSES] = {};
    double ms[WNNC_PROF_CLASSES] = {};
    cudaEvent_t get();
    void collect();       // synchronise pending records and accumulate
    void reset();
    ~Profiler();
};

// Brackets the launches issued while it lives with two events (when on).
struct ProfScope {
    Profiler* p;
    int cls;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(Profiler* p_, int cls_, cudaStream_t s_);
    ~ProfScope();
};

// ---------------------------------------------------------------------------
// The tree object behind the opaque wnnc_tree handle.
// ---------------------------------------------------------------------------
struct Tree {
    int64_t n = 0;
    wnnc_tree_params params{};
    double center[3] = {0, 0, 0};
    double scale = 1.0;
    int device = 0;

    // sorted sources
    uint64_t* keys = nullptr;     // Morton keys, sorted
    double* xs = nullptr;         // normalised coordinates, sorted (n x 3), build only

    // nodes, breadth-first
    int nnodes = 0, nleaves = 0, depth_reached = 0;
    int* node_start = nullptr;
    int* node_count = nullptr;
    int* node_parent = nullptr;
    int* node_child0 = nullptr;
    int* node_nchild = nullptr;
    int* node_depth = nullptr;
    int* level_off = nullptr;     // host: first node of each level, [levels+1]
    int nlevels = 0;
    int nmom_mid = 0;             // nodes of kMomSmall+1 .. kMomDirect points, and leaves of more
    int* mom_mid = nullptr;       // their ids
    int nmom_top = 0;             // inner nodes of more than kMomDirect points
    int* mom_top = nullptr;       // their ids
    int2* mom_top_rng = nullptr;  // per top node: its range of mom_front
    int* mom_front = nullptr;     // the non-top nodes whose parent is a top node, by first point
    double* node_lo = nullptr;    // tight bounding boxes (build)
    double* node_hi = nullptr;
    float4* node_lof = nullptr;   // the same boxes rounded outward to float (traversal pre-test)
    float4* node_hif = nullptr;
    float4* node_cell = nullptr;  // cell centre (exact) + width
    float4* node_cent = nullptr;  // point centroid - cell centre
    int* leaf_of = nullptr;       // sorted point -> leaf node

    // the points as their own targets
    TargetSet self;

    // transposed lists (adjoint, rep_mode 1)
    int* tfar_off = nullptr;      // [nnodes+1]
    int* tfar_ent = nullptr;      // far-entry index (position in self.far_id), grouped by node; with
                                  // local expansions class << 30 | id: 0 the entry, 1 (expanded about
                                  // a group) the group, 2 (about a cluster) the cluster
    int nach = 0;                 // source chunks of the adjoint near part (kAdjChunk points each)
    int* tnear_off = nullptr;     // [nach+1], per source chunk
    // per (source chunk, target group): (near slot of the first point of the
    // chunk in the group's near lists, mask of those points)
    int2* tnear_ent = nullptr;
    int64_t tnear_entries = 0;
    // Near slots: the (target group, source point) incidences of the near
    // lists, numbered group by group along each group's ranges.  rng_slot[q]
    // is the slot of the first point of near range q.
    int* rng_slot = nullptr;      // [near_ranges+1]
    int64_t near_slots = 0;
    WorkList adj_far_work;        // items over the far lists (per target group)
    WorkList adj_pair_work;       // items over the near ranges (per target group)
    WorkList adj_near_work;       // items over the transposed near entries (per source chunk)

    // work buffers (sized at build)
    float4* mu_a = nullptr;       // sorted normalised mu (two buffers)
    float4* mu_b = nullptr;
    float4* r_s = nullptr;        // sorted residual direction r
    float4* g_mu = nullptr;       // G(mu) and G(r) of the fused iteration (sorted, normalised)
    float4* g_r = nullptr;
    float* s_s = nullptr;         // sorted scalar field (s or adjoint input)
    float* area_s = nullptr;      // sorted areas (rescale mode 1)
    float4* mom = nullptr;        // node moments: (nu_x, nu_y, nu_z, sum|nu|)
    float4* mom_r = nullptr;      // node moments of the step direction r (same layout)
    float4* node_rep = nullptr;   // representative offset from cell centre, per call
    float4* contrib = nullptr;    // per far entry contribution (adjoint)
    float4* near_contrib = nullptr;   // per near slot contribution (adjoint)
    float4* vnode = nullptr;      // per node far sum (adjoint)
    float4* mom_x = nullptr;      // node weighted offsets (rep_mode 0): sum |nu| (x - cell), -
    double* dmom = nullptr;       // double node sums (moments_fp64), 8 per node
    // first-order far field (far_order 1)
    float4* mom_dip = nullptr;    // per node 2 float4: (Sxx, Syy, Szz, Sxy), (Sxz, Syz, tr S, 0) of mu
    float4* mom_dip_r = nullptr;  // the same of the step direction r
    float4* dip_corr = nullptr;   // per sorted target: first-order far terms (G x, y, z, A), sum units,
                                  // or the terms of the expanded far entries (local_theta > 0)
    // local expansions (local_theta > 0)
    float4* node_abs = nullptr;   // per node: point centroid in normalised coordinates (float)
    float4* local_rec = nullptr;  // per node, 32 bytes, rebuilt per call: (centroid, M_x), (M_y, M_z, 0, 0)
    float4* gadj = nullptr;       // per group, rebuilt per adjoint call: (c_g, rho_g), (D, S)
    float4* cadj = nullptr;       // per cluster, rebuilt per adjoint call: (c_C, rho_C), (D, S)
    float4* contrib_h0 = nullptr; // per far entry: sum s HPhi, (xx, yy, zz, -) and (xy, xz, yz, -)
    float4* contrib_h1 = nullptr;
    float4* hnode0 = nullptr;     // per node: the entries' sums of s HPhi (same two parts)
    float4* hnode1 = nullptr;
    double* partials = nullptr;   // per-group partial sums (3 x max(ngroups, nchunks, nach))
    double* red = nullptr;        // first-stage sums of the partials (3 x 256)
    unsigned* red_ticket = nullptr;   // blocks of the first stage done (the last one finishes)
    float4* part_acc = nullptr;   // scratch: partial sums of cut groups, 32 per slot
    int part_slots = 0;
    double* scalars = nullptr;    // device scalars: [0]=E [1]=rr [2]=qq [3]=alpha
    int* err_flag = nullptr;      // device error flags
    // a second stream for the adjoint's near pair sums, which overlap its far path, and
    // for the expanded far entries, which overlap the gather (its sums wait in gather_raw)
    cudaStream_t aux = nullptr;
    float4* gather_raw = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    Profiler prof;
};

// scan / sort primitives (scan_sort.cu)
void exclusive_scan_i32(const int* in, int* out, int64_t n, cudaStream_t s);   // out[n] = total
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on key bits [lo_bit, bits).  When
// the input is already ordered by the bits below lo_bit among equal higher
// bits (e.g. an index appended in ascending order), stability makes the result
// the same as a sort on all the low `bits` bits.
void radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s, int lo_bit = 0);
// Single-pass scans and sorts count a bounded wait that gave up in a device
// word: wait_timeouts_async queues its copy into *host (read it after a
// synchronisation of s); check_wait_timeouts clears it and fails with
// WNNC_ETIMEOUT when the value read is non-zero.
void wait_timeouts_async(unsigned* host, cudaStream_t s);
void check_wait_timeouts(unsigned seen, cudaStream_t s);
// One block of the single-pass scan whose look-back wait runs out (diagnostic).
void selftest_wait_timeout(cudaStream_t s);
// off[g] = first index i with (keys[i] >> shift) >= g, for g in [0, ng]; keys sorted.
void segment_offsets_hi32(const uint64_t* keys, int64_t n, int* off, int ng, cudaStream_t s, int shift = 32);

// tree build (tree_build.cu)
void build_tree(Tree& t, const float* pts, cudaStream_t s);
// self = the tree's own points as targets (groups cut at Morton jumps; the
// tree's sorted keys, coordinates and permutation `self_perm` are reused);
// otherwise fixed 32-target groups.
// Per-node data of the local expansions (local_theta > 0): the absolute
// centroids, computed once after the build.
void local_setup(Tree& t, cudaStream_t s);

// after_far (optional) runs on the host once the far lists are final (the
// work queued on s before it has produced them): the tree build forks the
// transposed lists onto a second stream there.
void build_target_set(const Tree& t, TargetSet& ts, const double* yn_unsorted, int64_t m, bool self,
                      cudaStream_t s, const int64_t* self_perm = nullptr,
                      const std::function<void()>& after_far = nullptr);
void free_target_set(TargetSet& ts);
void free_tree(Tree& t);

// operators (operators.cu)
enum Op : int { kOpA = 0, kOpG = 1, kOpATpaper = 2, kOpAG = 3 };
void moments(Tree& t, const float4* nu_sorted_vec, const float* nu_sorted_scalar, int rep_mode, float4* out,
             cudaStream_t s);
void eval_w(Tree& t, const float* mu, float w, float* out, cudaStream_t s);
void eval_grad(Tree& t, const float* mu, float w, float* out, cudaStream_t s);
void eval_adjoint(Tree& t, const float* sv, float w, float* out, cudaStream_t s);
void eval_at(Tree& t, const float* mu, const float* q, int64_t m, float w, int grad, float* out,
             cudaStream_t s);
void iterate(Tree& t, float* mu_inout, const float* area, const wnnc_iter_params& p,
             cudaStream_t s, float* stats);

// k nearest neighbours and patch features (knn.cu)
void knn16(Tree& t, int* idx_out, float* feat_out, cudaStream_t s);

// point-patch MLP of the warm start (mlp.cu)
struct Mlp {
    int64_t max_batch = 0;
    float* params = nullptr;   // FP32 master parameters (BF16-rounded when read)
    float* m = nullptr;        // Adam moments
    float* v = nullptr;
    float* grad = nullptr;
    float* h1 = nullptr;       // [B][128] activations (after ReLU)
    float* h2 = nullptr;
    float* h3 = nullptr;
    float* out = nullptr;      // [B][3]
    float* d3 = nullptr;       // [B][128] gradients w.r.t. pre-activations
    float* d2 = nullptr;
    float* d1 = nullptr;
    float* dout = nullptr;     // [B][3]
    float* part = nullptr;     // weight-gradient partials [nchunk][params]
    double* lpart = nullptr;   // loss partials
    int64_t step = 0;
    int loss_mode = 0;         // 0: 1 - c (signed), 1: 1 - c^2 (sign-free); c = (v/|v|).label
};
int mlp_param_count();
double probe_fp32(cudaStream_t s);
void mlp_alloc(Mlp& m, int64_t max_batch);
void mlp_free(Mlp& m);
void mlp_forward(Mlp& m, const float* x, int64_t B, float* y, cudaStream_t s);
void mlp_grad(Mlp& m, const float* x, const float* label, int64_t B, float* loss_dev, cudaStream_t s);
void mlp_adam(Mlp& m, float lr, cudaStream_t s);
void warm_init(const float* dir, const float* ref, int64_t n, float area, float* mu, cudaStream_t s);

}  // namespace wnnc
