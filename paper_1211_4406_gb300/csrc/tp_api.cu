// tp_api.cu -- the C-ABI of libtreepm_sr.so (declared in include/treepm_sr.h):
// tree lifecycle, build orchestration, force / adjoint dispatch, parity
// exports, leapfrog helpers and the FMA peak microbenchmark.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "tp_common.cuh"
#include "tp_nvtx.h"

namespace tp {
void build_keys_sort_gather(TreeDev &T, const double *pos, const double *mass, uint64_t *key2,
                            uint32_t *perm2, void *radix_tmp, cudaStream_t s);
void build_topology(TreeDev &T, uint32_t *nch, uint32_t *ofs, int32_t *cb, void *scan_tmp, cudaStream_t s);
void build_boxes(TreeDev &T, cudaStream_t s);
void build_masses(TreeDev &T, cudaStream_t s);
void build_group_starts(TreeDev &T, uint32_t *flag, uint32_t *gofs, void *scan_tmp, cudaStream_t s);
void build_groups(TreeDev &T, const uint32_t *flag, const uint32_t *gofs, cudaStream_t s);
void walk_top_count(TreeDev &T, int32_t split, void *scan_tmp, cudaStream_t s);
void walk_items(TreeDev &T, int32_t split, void *scan_tmp, cudaStream_t s);
void walk_expand(TreeDev &T, unsigned long long *counter, void *scan_tmp, cudaStream_t s);
void walk_write(TreeDev &T, cudaStream_t s);
void walk_top_scan(TreeDev &T, void *scan_tmp, cudaStream_t s);
void vjp_begin(TreeDev &T, double *gs, double *ncot, cudaStream_t s);
void vjp_pairs_f32(TreeDev &T, const float *cot, double *gs, double *ncot, int32_t *queue, const int32_t *order,
                   int64_t G, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int adj_entries);
void vjp_pairs_f64(TreeDev &T, const double *cot, double *gs, double *ncot, int32_t *queue,
                   const int32_t *order, int64_t G, cudaStream_t s);
void vjp_end(TreeDev &T, double *grad, double *gs, double *ncot, int32_t *leaf_of, cudaStream_t s);
void force_vjp_pairs_f32(TreeDev &T, float *acc, const float *cot, double *gs, double *ncot, int32_t *queue,
                         const int32_t *order, int64_t G, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                         int adj_entries);
void lpt_order(TreeDev &T, uint64_t *key, uint32_t *val, uint64_t *key2, uint32_t *val2,
               void *radix_tmp, cudaStream_t s);
void list_stats(TreeDev &T, unsigned long long *inter, int32_t *max_nj, cudaStream_t s);
void count_useful(TreeDev &T, unsigned long long *useful, cudaStream_t s);
void pair_forward_f32(TreeDev &T, float *acc, int32_t *queue, const int32_t *order, int64_t G,
                      cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int fwd_particles);
void pair_forward_f64(TreeDev &T, double *acc, int64_t G, cudaStream_t s);
void vjp_f32(TreeDev &T, const float *cot, double *grad, double *gs, double *ncot, int32_t *leaf_of,
             int32_t *queue, const int32_t *order, int64_t G, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
             int adj_entries);
void vjp_f64(TreeDev &T, const double *cot, double *grad, double *gs, double *ncot, int32_t *leaf_of,
             int32_t *queue, const int32_t *order, int64_t G, cudaStream_t s);
}  // namespace tp

static std::atomic<long long> g_launches{0};
extern "C" void tp_count_launch(void) { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

// Device allocations of one tree, freed together.
struct Pool {
    std::vector<void *> ptrs;
    bool ok = true;
    template <class T>
    T *get(size_t count)
    {
        void *p = nullptr;
        if (count == 0) count = 1;
        if (cudaMalloc(&p, sizeof(T) * count) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    void release()
    {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
        ok = true;
    }
};

uint64_t sat_u64(double v)
{
    if (!(v > 0.0)) return 0ull;
    if (v >= 18446744073709551615.0) return ~0ull;
    return (uint64_t)v;
}

BoxPrm make_box(const tp_params &p, int64_t first, int64_t count)
{
    BoxPrm b;
    std::memset(&b, 0, sizeof(b));
    b.G = p.G; b.eps = p.eps; b.rcut = p.r_cut; b.theta = p.theta;
    volatile double rc = p.r_cut, ep = p.eps, th = p.theta;
    b.rc2 = rc * rc;
    b.eps2 = ep * ep;
    b.th2 = th * th;
    const double k = 2.0 / p.r_cut;
    b.eps2s = (float)((k * p.eps) * (k * p.eps));
    b.scale = (float)(k * 5.421010862427522e-20);   // k * 2^-64
    b.gk2 = p.G * k * k;
    b.scale_d = 5.421010862427522e-20;
    const double E = TP_FILTER_SLACK;
    const double R = p.r_cut * 4294967296.0;
    b.T_hi = sat_u64(std::ceil((R + E) * (R + E))) + 1;
    b.T_lo = R > E + 1.0 ? sat_u64(std::floor((R - E) * (R - E)) - 1.0) : 0ull;
    for (int L = 0; L < TP_NLEVELS; L++) {
        if (!(p.theta > 0.0)) {
            b.TB_lo[L] = ~0ull;
            b.TB_hi[L] = ~0ull;
            continue;
        }
        const double lam = std::ldexp(1.0, 32 - L) / p.theta;
        const double hi = std::ceil((lam + E) * (lam + E)) + 1.0;
        b.TB_hi[L] = hi >= 18446744073709551615.0 ? ~0ull : sat_u64(hi);
        b.TB_lo[L] = lam > E + 1.0 ? sat_u64(std::floor((lam - E) * (lam - E)) - 1.0) : 0ull;
    }
    b.n_crit = p.n_crit;
    b.n_leaf = p.n_leaf;
    b.first = first;
    b.count = count;
    b.inv_n = count > 0 ? 1.0 / (double)count : 0.0;
    return b;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Events of the side stream: after the gather, after the topology, after the
// node boxes, after the monopoles, before and after the LPT order.
enum { kEvGather, kEvTopology, kEvBoxes, kEvMasses, kEvLists, kEvOrder, kSideEvents };

struct tp_tree {
    int64_t n = 0;
    int32_t nbox = 0;
    int32_t precision = TP_FP32;
    std::vector<int64_t> box_off;
    std::vector<tp_params> prm;
    cudaStream_t last = nullptr;
    // allocations: base (particles, workspace), nodes, groups, walk items, lists
    Pool base, nodes, groups, items, pad, lists;
    int32_t split = 1024;             // largest subtree a single walk task expands
    TreeDev D;
    // scratch
    uint64_t *key2 = nullptr;
    uint32_t *perm2 = nullptr;
    void *radix_tmp = nullptr, *scan_tmp = nullptr;
    uint32_t *flag = nullptr, *gofs = nullptr;
    uint32_t *nch = nullptr, *nofs = nullptr;
    int32_t *cbnd = nullptr;          // [7 cap_nodes] inner child bounds of one level's nodes
    int32_t *queue = nullptr;
    int32_t *order = nullptr;         // groups in LPT order for the work queue
    uint64_t *lpt_key = nullptr, *lpt_key2 = nullptr;
    uint32_t *lpt_val2 = nullptr;
    void *lpt_tmp = nullptr;
    double *gs = nullptr, *ncot = nullptr;
    unsigned long long *d_inter = nullptr, *d_useful = nullptr;
    int32_t *d_maxnj = nullptr;
    // host copies of the sizes (valid after a synchronising build)
    int64_t h_nodes = 0, h_groups = 0, h_items = 0, h_pad = 0, h_entries = 0;
    // chunked mode: windows [first group, group count) with lists of bounded size
    bool chunked = false, force_chunked = false, windows_stale = true;
    std::vector<int64_t> win_first, win_count, win_xitems;
    int64_t *d_wsz = nullptr;         // [kMaxWindows] device copies of the window sizes
    int64_t *d_etot = nullptr;        // entries summed over the windows
    // tile shapes of the FP32 pair kernels (tp_tree_set_tile)
    int32_t fwd_particles = 2, adj_entries = 4;
    // kernel timing: events around the main forward / adjoint kernel launches
    bool ktiming = false, kf_rec = false, kv_rec = false;
    cudaEvent_t kev[4] = {nullptr, nullptr, nullptr, nullptr};
    // a second stream for the build steps that do not depend on each other
    // (fork/join by events, so the calls stay ordered on the caller's stream
    // and capture into one graph): kSideEvents events, see side_fork/side_join
    cudaStream_t side = nullptr;
    cudaEvent_t sev[kSideEvents] = {};
};

// Scratch of n int32 for the adjoint's epilogue (each particle's leaf): the
// group-start flags, which only a build uses.
static int32_t *leaf_scratch(tp_tree *t) { return reinterpret_cast<int32_t *>(t->flag); }

// The side stream starts after everything issued on s so far.
static void side_fork(tp_tree *t, cudaStream_t s, int ev)
{
    cudaEventRecord(t->sev[ev], s);
    cudaStreamWaitEvent(t->side, t->sev[ev], 0);
}

// s continues after everything issued on the side stream so far.
static void side_join(tp_tree *t, cudaStream_t s, int ev)
{
    cudaEventRecord(t->sev[ev], t->side);
    cudaStreamWaitEvent(s, t->sev[ev], 0);
}

static tp_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return TP_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA;
}

static bool alloc_nodes(tp_tree *t, int64_t cap)
{
    Pool &P = t->nodes;
    P.release();
    TreeDev &D = t->D;
    D.cap_nodes = cap;
    size_t c = (size_t)cap;
    D.first = P.get<int32_t>(c); D.count = P.get<int32_t>(c); D.child = P.get<int32_t>(c);
    D.nchild = P.get<int32_t>(c); D.parent = P.get<int32_t>(c); D.skip = P.get<int32_t>(c);
    D.nbx = P.get<int32_t>(c); D.level = P.get<uint8_t>(c);
    D.M = P.get<double>(c); D.Sx = P.get<double>(c); D.Sy = P.get<double>(c); D.Sz = P.get<double>(c);
    D.comx = P.get<double>(c); D.comy = P.get<double>(c); D.comz = P.get<double>(c);
    D.lox = P.get<double>(c); D.loy = P.get<double>(c); D.loz = P.get<double>(c);
    D.hix = P.get<double>(c); D.hiy = P.get<double>(c); D.hiz = P.get<double>(c);
    D.cenx = P.get<double>(c); D.ceny = P.get<double>(c); D.cenz = P.get<double>(c);
    D.hfx = P.get<double>(c); D.hfy = P.get<double>(c); D.hfz = P.get<double>(c);
    D.cX = P.get<uint64_t>(c); D.cY = P.get<uint64_t>(c); D.cZ = P.get<uint64_t>(c);
    D.nsrc = P.get<SrcRec>(c);
    D.wn = P.get<WNode>(c);
    t->nch = P.get<uint32_t>(c);
    t->nofs = P.get<uint32_t>(c > 1024 ? c : 1024);   // also the topology passes' block sums (608 blocks)
    t->cbnd = P.get<int32_t>(7 * c);
    t->ncot = P.get<double>(3 * c);
    return P.ok;
}

static bool alloc_groups(tp_tree *t, int64_t cap)
{
    Pool &P = t->groups;
    P.release();
    TreeDev &D = t->D;
    D.cap_groups = cap;
    size_t c = (size_t)cap;
    D.gfirst = P.get<int32_t>(c); D.gcount = P.get<int32_t>(c); D.gbox = P.get<int32_t>(c);
    D.gcx = P.get<double>(c); D.gcy = P.get<double>(c); D.gcz = P.get<double>(c);
    D.ghx = P.get<double>(c); D.ghy = P.get<double>(c); D.ghz = P.get<double>(c);
    D.gux = P.get<uint32_t>(c); D.guy = P.get<uint32_t>(c); D.guz = P.get<uint32_t>(c);
    D.ghux = P.get<uint32_t>(c); D.ghuy = P.get<uint32_t>(c); D.ghuz = P.get<uint32_t>(c);
    D.gX = P.get<uint64_t>(c); D.gY = P.get<uint64_t>(c); D.gZ = P.get<uint64_t>(c);
    D.loff = P.get<int64_t>(c + 1);
    D.lcnt = P.get<int32_t>(c);
    D.gpad = P.get<int32_t>(c);
    D.icnt = P.get<int32_t>(c);
    D.kscr = (int32_t)(kTopScratchTotal / (int64_t)(c > 0 ? c : 1) < kTopScratch
                           ? kTopScratchTotal / (int64_t)(c > 0 ? c : 1) : kTopScratch);
    D.iscr = P.get<int32_t>(c * (size_t)D.kscr);
    D.ioff = P.get<int64_t>(c);
    // work items: the groups' first chunks and up to cap_xitems further ones
    const size_t cw = c + (size_t)D.cap_xitems;
    t->lpt_key = P.get<uint64_t>(cw);
    t->lpt_key2 = P.get<uint64_t>(cw);
    t->order = reinterpret_cast<int32_t *>(P.get<uint32_t>(cw));
    t->lpt_val2 = P.get<uint32_t>(cw);
    t->lpt_tmp = P.get<char>(tp::radix_tmp_bytes((int64_t)cw));
    return P.ok;
}

static bool alloc_items(tp_tree *t, int64_t cap)
{
    Pool &P = t->items;
    P.release();
    TreeDev &D = t->D;
    D.cap_items = cap;
    size_t c = (size_t)cap;
    D.item = P.get<int32_t>(c); D.igrp = P.get<int32_t>(c); D.icnt2 = P.get<int32_t>(c);
    D.ipos = P.get<int64_t>(c);
    D.ibpos = P.get<int64_t>(c);
    D.ibound = P.get<int32_t>(c);
    return P.ok;
}

static bool alloc_pad(tp_tree *t, int64_t cap)
{
    Pool &P = t->pad;
    P.release();
    t->D.cap_pad = cap;
    t->D.pent = P.get<int32_t>((size_t)cap);
    return P.ok;
}

static bool alloc_lists(tp_tree *t, int64_t cap)
{
    Pool &P = t->lists;
    P.release();
    t->D.cap_entries = cap;
    t->D.ent = P.get<int32_t>((size_t)cap);
    t->D.rec = P.get<float4>((size_t)cap);
    return P.ok;
}

template <class T>
static std::vector<T> fetch(const T *d, int64_t n)
{
    std::vector<T> h((size_t)(n > 0 ? n : 0));
    if (n > 0) cudaMemcpy(h.data(), d, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost);
    return h;
}

static tp_status validate(const tp_params &p)
{
    if (!(p.r_cut > 0.0 && p.r_cut < 0.5)) return TP_ERR_INVALID_ARG;
    if (!(p.eps >= 0.0) || !std::isfinite(p.eps)) return TP_ERR_INVALID_ARG;
    if (!(p.theta >= 0.0) || !std::isfinite(p.theta)) return TP_ERR_INVALID_ARG;
    if (!std::isfinite(p.G)) return TP_ERR_INVALID_ARG;
    if (p.n_crit < 1 || p.n_crit > 4096 || p.n_leaf < 1 || p.n_leaf > 64) return TP_ERR_INVALID_ARG;
    if (p.precision != TP_FP32 && p.precision != TP_FP64) return TP_ERR_INVALID_ARG;
    if (p.flags & ~(TP_FLAG_CHUNKED | TP_FLAG_XI_SOFTENED | TP_FLAG_RSQRT_REFINED)) return TP_ERR_INVALID_ARG;
    if ((p.flags & TP_FLAG_RSQRT_REFINED) && p.precision != TP_FP32) return TP_ERR_INVALID_ARG;
    return TP_OK;
}

__global__ void k_clamp_groups(TreeDev T)
{
    if (*T.n_groups > T.cap_groups) {
        tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
        *T.n_groups = T.cap_groups;
    }
}

__global__ void k_check_items(TreeDev T)
{
    if (*T.n_items > T.cap_items) tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
}

__global__ void k_check_pad(TreeDev T)
{
    if (*T.n_pad > T.cap_pad) tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
}

__global__ void k_check_entries(TreeDev T)
{
    if (*T.n_entries > T.cap_entries) tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
    if (*T.n_groups > T.cap_groups) tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
}

// ---------------------------------------------------------------------------
// Chunked mode.  A window of consecutive groups is evaluated through a view of
// the tree whose group arrays start at the window's first group and whose
// group count is the window's size, so every walk and pair kernel runs on it
// unchanged, with its items, padded slots and lists reusing the same buffers.
constexpr int64_t kWindowSlots = 1ll << 29;  // padded-slot budget of one window
constexpr double kSlotBytes = 4.0 + 4.0 + 16.0;   // per padded slot: slot, entry id, entry record
constexpr int kMaxWindows = 1 << 16;

static TreeDev window_view(const TreeDev &D, int64_t g0, int64_t ng, int64_t *d_ng, int64_t nx)
{
    TreeDev V = D;
    V.cap_xitems = nx < D.cap_xitems ? nx : D.cap_xitems;   // the window's further chunks
    V.gfirst += g0; V.gcount += g0; V.gbox += g0;
    V.gcx += g0; V.gcy += g0; V.gcz += g0; V.ghx += g0; V.ghy += g0; V.ghz += g0;
    V.gux += g0; V.guy += g0; V.guz += g0; V.ghux += g0; V.ghuy += g0; V.ghuz += g0;
    V.gX += g0; V.gY += g0; V.gZ += g0;
    V.gpad += g0; V.loff += g0; V.lcnt += g0; V.icnt += g0; V.ioff += g0;
    V.iscr += g0 * D.kscr;
    V.n_groups = d_ng;
    V.cap_groups = ng;
    return V;
}

// Greedy windows over the groups' item counts and padded-slot bounds (from
// the count pass of the top walk): consecutive groups while both sums stay
// within the budgets; a group that alone exceeds them gets a window of its own
// (its walk then latches TP_ERR_LIST_OVERFLOW).  Synchronises.
static tp_status plan_windows(tp_tree *t, cudaStream_t s, int64_t slot_budget, int64_t item_budget,
                              int64_t *max_slots, int64_t *max_items)
{
    TreeDev &D = t->D;
    int64_t G = 0;
    tp_status e = cuda_status(cudaMemcpyAsync(&G, D.n_groups, sizeof(G), cudaMemcpyDeviceToHost, s));
    if (e == TP_OK) e = cuda_status(cudaStreamSynchronize(s));
    if (e != TP_OK) return e;
    if (G > D.cap_groups) G = D.cap_groups;
    std::vector<int32_t> ic((size_t)(G > 0 ? G : 1)), gp((size_t)(G > 0 ? G : 1)), gc((size_t)(G > 0 ? G : 1));
    if (G > 0) {
        e = cuda_status(cudaMemcpy(ic.data(), D.icnt, sizeof(int32_t) * G, cudaMemcpyDeviceToHost));
        if (e == TP_OK) e = cuda_status(cudaMemcpy(gp.data(), D.gpad, sizeof(int32_t) * G, cudaMemcpyDeviceToHost));
        if (e == TP_OK) e = cuda_status(cudaMemcpy(gc.data(), D.gcount, sizeof(int32_t) * G, cudaMemcpyDeviceToHost));
        if (e != TP_OK) return e;
    }
    t->win_first.clear();
    t->win_count.clear();
    t->win_xitems.clear();
    int64_t g0 = 0, slots = 0, items = 0, xitems = 0, ms = 0, mi = 0;
    for (int64_t g = 0; g <= G; g++) {
        const bool close = g == G || (g > g0 && (slots + gp[g] > slot_budget || items + ic[g] > item_budget));
        if (close && g > g0) {
            t->win_first.push_back(g0);
            t->win_count.push_back(g - g0);
            t->win_xitems.push_back(xitems);
            ms = slots > ms ? slots : ms;
            mi = items > mi ? items : mi;
            g0 = g;
            slots = items = xitems = 0;
        }
        if (g < G) {
            slots += gp[g];
            items += ic[g];
            if (gc[g] > kWorkChunk) xitems += (gc[g] - 1) / kWorkChunk;   // chunks after the first
        }
    }
    if ((int64_t)t->win_count.size() > kMaxWindows) return TP_ERR_LIST_OVERFLOW;
    if (!t->win_count.empty()) {
        e = cuda_status(cudaMemcpyAsync(t->d_wsz, t->win_count.data(), sizeof(int64_t) * t->win_count.size(),
                                        cudaMemcpyHostToDevice, s));
        if (e != TP_OK) return e;
    }
    if (max_slots) *max_slots = ms;
    if (max_items) *max_items = mi;
    t->windows_stale = false;
    return TP_OK;
}

__global__ void k_add_entries(TreeDev V, int64_t *tot) { *tot += *V.n_entries; }

// Node boxes and walk records, then the monopoles, on the side stream once
// the topology issued on s is final: the walk waits for the boxes only
// (kEvBoxes), the compaction and every later use for the monopoles
// (kEvMasses), which thus run beside the walk.
static void fork_moments(tp_tree *t, cudaStream_t s)
{
    side_fork(t, s, kEvTopology);
    tp::build_boxes(t->D, t->side);
    cudaEventRecord(t->sev[kEvBoxes], t->side);
    tp::build_masses(t->D, t->side);
    cudaEventRecord(t->sev[kEvMasses], t->side);
}

// The lists and their records (k_compact, which reads the monopoles' source
// records), and beside them on the side stream the LPT order of the work
// items, which needs only the list counts.
static void write_and_order(tp_tree *t, TreeDev &V, cudaStream_t s)
{
    cudaStreamWaitEvent(s, t->sev[kEvMasses], 0);
    side_fork(t, s, kEvLists);
    tp::lpt_order(V, t->lpt_key, reinterpret_cast<uint32_t *>(t->order), t->lpt_key2, t->lpt_val2,
                  t->lpt_tmp, t->side);
    tp::walk_write(V, s);
    side_join(t, s, kEvOrder);
}

// The walk of one window: items, tasks, lists and records, LPT order; list
// statistics accumulate into the tree's counters.
static void walk_window(tp_tree *t, TreeDev &V, cudaStream_t s)
{
    tp::walk_top_scan(V, t->scan_tmp, s);
    TP_LAUNCH(k_check_items, 1, 1, 0, s, V);
    tp::walk_items(V, t->split, t->scan_tmp, s);
    TP_LAUNCH(k_check_pad, 1, 1, 0, s, V);
    tp::walk_expand(V, reinterpret_cast<unsigned long long *>(t->queue + 2), t->scan_tmp, s);
    TP_LAUNCH(k_check_entries, 1, 1, 0, s, V);
    write_and_order(t, V, s);
    tp::list_stats(V, t->d_inter, t->d_maxnj, s);
    TP_LAUNCH(k_add_entries, 1, 1, 0, s, V, t->d_etot);
}

static void reset_list_stats(tp_tree *t, cudaStream_t s)
{
    cudaMemsetAsync(t->d_inter, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(t->d_maxnj, 0, sizeof(int32_t), s);
    cudaMemsetAsync(t->d_etot, 0, sizeof(int64_t), s);
}

// Runs `body(view)` for every window (planning them first when the positions
// changed since they were planned).
template <class F>
static tp_status for_each_window(tp_tree *t, cudaStream_t s, F body)
{
    if (t->windows_stale) {
        tp_status e = plan_windows(t, s, t->D.cap_pad, t->D.cap_items, nullptr, nullptr);
        if (e != TP_OK) return e;
    }
    reset_list_stats(t, s);
    for (size_t w = 0; w < t->win_count.size(); w++) {
        TreeDev V = window_view(t->D, t->win_first[w], t->win_count[w], t->d_wsz + w, t->win_xitems[w]);
        walk_window(t, V, s);
        body(V);
    }
    return TP_OK;
}

// The allocating build's walk in chunked mode: plan windows of about
// `budget` padded slots, size the item / slot / list buffers for the largest,
// and walk every window once (capacity check and statistics).
static tp_status build_chunked(tp_tree *t, cudaStream_t s, int64_t budget)
{
    TreeDev &D = t->D;
    int64_t ms = 0, mi = 0;
    tp_status e = plan_windows(t, s, budget, INT64_MAX, &ms, &mi);
    if (e != TP_OK) return e;
    if (mi > D.cap_items || D.item == nullptr)
        if (!alloc_items(t, mi + 1024)) return TP_ERR_OOM;
    if (ms > D.cap_pad || D.pent == nullptr)
        if (!alloc_pad(t, ms + 1024)) return TP_ERR_OOM;
    if (ms > D.cap_entries || D.ent == nullptr)
        if (!alloc_lists(t, ms + 1024)) return TP_ERR_OOM;
    e = for_each_window(t, s, [](TreeDev &) {});
    if (e != TP_OK) return e;
    return cuda_status(cudaStreamSynchronize(s));
}

// Launch everything after the keys: topology, groups, walk.  With `sync`
// set, sizes are read back and buffers (re)allocated to fit.
static tp_status run_build(tp_tree *t, const double *pos, const double *mass, cudaStream_t s, bool sync)
{
    TreeDev &D = t->D;
    NvtxRange construction("tree construction");
    cudaMemsetAsync(D.status, 0, sizeof(int32_t), s);
    cudaMemsetAsync(D.n_ambig, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(D.n_general, 0xff, sizeof(unsigned long long), s);   // counted again by the LPT pass
    tp::build_keys_sort_gather(D, pos, mass, t->key2, t->perm2, t->radix_tmp, s);
    // Side stream: the refit reference (the sorted positions of the latest
    // tree build), then the boxes and monopoles once the topology is final
    // (fork_moments); the groups go on beside them on s.
    side_fork(t, s, kEvGather);
    if (D.n > 0) {
        cudaMemcpyAsync(D.rx, D.x, sizeof(double) * (size_t)D.n, cudaMemcpyDeviceToDevice, t->side);
        cudaMemcpyAsync(D.ry, D.y, sizeof(double) * (size_t)D.n, cudaMemcpyDeviceToDevice, t->side);
        cudaMemcpyAsync(D.rz, D.z, sizeof(double) * (size_t)D.n, cudaMemcpyDeviceToDevice, t->side);
    }
    bool moments = false;
    for (int attempt = 0;; attempt++) {
        tp::build_topology(D, t->nch, t->nofs, t->cbnd, t->scan_tmp, s);
        if (!sync) {                          // no host check can send the topology round again
            fork_moments(t, s);
            moments = true;
        }
        tp::build_group_starts(D, t->flag, t->gofs, t->scan_tmp, s);
        if (!sync) break;
        int32_t st = 0;
        cudaMemcpyAsync(&st, D.status, sizeof(st), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&t->h_nodes, D.n_nodes, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&t->h_groups, D.n_groups, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        tp_status e = cuda_status(cudaStreamSynchronize(s));
        if (e != TP_OK) return e;
        if (st == TP_ERR_NONFINITE) return TP_ERR_NONFINITE;
        if (st == TP_ERR_LIST_OVERFLOW && attempt < 8) {
            if (!alloc_nodes(t, 2 * D.cap_nodes)) return TP_ERR_OOM;
            cudaMemsetAsync(D.status, 0, sizeof(int32_t), s);
            continue;
        }
        if (st != 0) return (tp_status)st;
        if (t->h_groups > D.cap_groups || D.gfirst == nullptr) {
            if (!alloc_groups(t, t->h_groups + t->h_groups / 4 + 64)) return TP_ERR_OOM;
        }
        break;
    }
    if (!moments) fork_moments(t, s);
    TP_LAUNCH(k_clamp_groups, 1, 1, 0, s, D);
    tp::build_groups(D, t->flag, t->gofs, s);
    cudaStreamWaitEvent(s, t->sev[kEvBoxes], 0);
    construction.end();
    NvtxRange traversal("tree traversal");
    // walk: top items per group, then subtree tasks, then the entries
    tp::walk_top_count(D, t->split, t->scan_tmp, s);
    if (!sync && t->chunked) {             // the next force/vjp call plans the windows
        cudaStreamWaitEvent(s, t->sev[kEvMasses], 0);
        t->windows_stale = true;
        return TP_OK;
    }
    if (sync) {
        // whole lists, or windows of them when they would not fit
        int64_t G = t->h_groups < D.cap_groups ? t->h_groups : D.cap_groups;
        std::vector<int32_t> gp((size_t)(G > 0 ? G : 1));
        if (G > 0) {
            tp_status e = cuda_status(cudaMemcpyAsync(gp.data(), D.gpad, sizeof(int32_t) * G,
                                                      cudaMemcpyDeviceToHost, s));
            if (e == TP_OK) e = cuda_status(cudaStreamSynchronize(s));
            if (e != TP_OK) return e;
        }
        int64_t total = 0, largest = 0;
        for (int64_t g = 0; g < G; g++) {
            total += gp[g];
            largest = gp[g] > largest ? gp[g] : largest;
        }
        // whole lists when their buffers take at most half of the free device memory
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            free_b = 0;
        }
        t->chunked = t->force_chunked || kSlotBytes * (double)total > 0.5 * (double)free_b;
        if (t->chunked) {
            int64_t budget = t->force_chunked ? total / 4 + 1 : kWindowSlots;
            return build_chunked(t, s, budget > largest ? budget : largest);
        }
    }
    if (sync) {
        tp_status e = cuda_status(cudaMemcpyAsync(&t->h_items, D.n_items, sizeof(int64_t),
                                                  cudaMemcpyDeviceToHost, s));
        if (e == TP_OK) e = cuda_status(cudaStreamSynchronize(s));
        if (e != TP_OK) return e;
        if (t->h_items > D.cap_items || D.item == nullptr) {
            if (!alloc_items(t, t->h_items + t->h_items / 4 + 1024)) return TP_ERR_OOM;
        }
    }
    TP_LAUNCH(k_check_items, 1, 1, 0, s, D);
    tp::walk_items(D, t->split, t->scan_tmp, s);
    if (sync) {
        tp_status e = cuda_status(cudaMemcpyAsync(&t->h_pad, D.n_pad, sizeof(int64_t),
                                                  cudaMemcpyDeviceToHost, s));
        if (e == TP_OK) e = cuda_status(cudaStreamSynchronize(s));
        if (e != TP_OK) return e;
        if (t->h_pad > D.cap_pad || D.pent == nullptr) {
            if (!alloc_pad(t, t->h_pad + t->h_pad / 4 + 1024)) return TP_ERR_OOM;
        }
    }
    TP_LAUNCH(k_check_pad, 1, 1, 0, s, D);
    tp::walk_expand(D, reinterpret_cast<unsigned long long *>(t->queue + 2), t->scan_tmp, s);
    if (sync) {
        tp_status e = cuda_status(cudaMemcpyAsync(&t->h_entries, D.n_entries, sizeof(int64_t),
                                                  cudaMemcpyDeviceToHost, s));
        if (e == TP_OK) e = cuda_status(cudaStreamSynchronize(s));
        if (e != TP_OK) return e;
        if (t->h_entries > D.cap_entries || D.ent == nullptr) {
            if (!alloc_lists(t, t->h_entries + t->h_entries / 4 + 1024)) return TP_ERR_OOM;
        }
    }
    TP_LAUNCH(k_check_entries, 1, 1, 0, s, D);
    write_and_order(t, D, s);
    return TP_OK;
}

extern "C" {

tp_status tp_build_tree_batched(const double *pos, const double *mass, const int64_t *box_offsets,
                                int32_t nbox, const tp_params *per_box, void *stream, tp_tree **out)
{
    if (!out || !box_offsets || !per_box || nbox < 1) return TP_ERR_INVALID_ARG;
    *out = nullptr;
    if (box_offsets[0] != 0) return TP_ERR_INVALID_ARG;
    for (int b = 0; b < nbox; b++) {
        if (box_offsets[b + 1] < box_offsets[b]) return TP_ERR_INVALID_ARG;
        if (validate(per_box[b]) != TP_OK) return TP_ERR_INVALID_ARG;
        if (per_box[b].precision != per_box[0].precision) return TP_ERR_INVALID_ARG;
        if ((per_box[b].flags ^ per_box[0].flags) & (TP_FLAG_XI_SOFTENED | TP_FLAG_RSQRT_REFINED))
            return TP_ERR_INVALID_ARG;
    }
    const int64_t n = box_offsets[nbox];
    if (n < 0 || n >= (1ll << 31) - 1) return TP_ERR_INVALID_ARG;
    if (n > 0 && !is_device_ptr(pos)) return TP_ERR_INVALID_ARG;
    if (mass && !is_device_ptr(mass)) return TP_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return TP_ERR_NO_DEVICE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    tp_tree *t = new tp_tree();
    t->n = n;
    t->nbox = nbox;
    t->precision = per_box[0].precision;
    t->box_off.assign(box_offsets, box_offsets + nbox + 1);
    t->prm.assign(per_box, per_box + nbox);
    for (int b = 0; b < nbox; b++)
        if (per_box[b].flags & TP_FLAG_CHUNKED) t->force_chunked = true;
    t->last = s;
    bool side_ok = cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &e : t->sev) side_ok = side_ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (!side_ok) {
        tp_tree_free(t);
        return TP_ERR_CUDA;
    }
    TreeDev &D = t->D;
    std::memset(&D, 0, sizeof(D));
    D.n = n;
    D.nbox = nbox;
    D.xi_soft = (per_box[0].flags & TP_FLAG_XI_SOFTENED) ? 1 : 0;
    D.rsq_refined = (per_box[0].flags & TP_FLAG_RSQRT_REFINED) ? 1 : 0;
    Pool &B = t->base;
    std::vector<BoxPrm> hb(nbox);
    for (int b = 0; b < nbox; b++)
        hb[b] = make_box(per_box[b], box_offsets[b], box_offsets[b + 1] - box_offsets[b]);
    BoxPrm *dbox = B.get<BoxPrm>(nbox);
    int64_t *dboff = B.get<int64_t>(nbox + 1);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    D.key = B.get<uint64_t>(nn); D.perm = B.get<uint32_t>(nn);
    t->key2 = B.get<uint64_t>(nn); t->perm2 = B.get<uint32_t>(nn);
    D.x = B.get<double>(nn); D.y = B.get<double>(nn); D.z = B.get<double>(nn); D.m = B.get<double>(nn);
    D.X = B.get<uint64_t>(nn); D.Y = B.get<uint64_t>(nn); D.Z = B.get<uint64_t>(nn);
    D.P32 = B.get<uint4>(nn);
    D.rx = B.get<double>(nn); D.ry = B.get<double>(nn); D.rz = B.get<double>(nn);
    D.psrc = B.get<SrcRec>(nn);
    t->radix_tmp = B.get<char>(tp::radix_tmp_bytes(n));
    t->scan_tmp = B.get<char>(tp::scan_tmp_bytes());
    t->flag = B.get<uint32_t>(nn); t->gofs = B.get<uint32_t>(nn);
    D.lstart = B.get<int64_t>(TP_NLEVELS + 1); D.lcount = B.get<int64_t>(TP_NLEVELS + 1);
    D.n_nodes = B.get<int64_t>(1); D.n_groups = B.get<int64_t>(1); D.n_entries = B.get<int64_t>(1);
    D.n_items = B.get<int64_t>(1);
    D.n_pad = B.get<int64_t>(1);
    D.n_ambig = B.get<unsigned long long>(1);
    D.n_general = B.get<unsigned long long>(1);
    // every further chunk of a group holds kWorkChunk particles of its own
    D.cap_xitems = n / kWorkChunk + 1;
    D.xitem = B.get<int2>((size_t)D.cap_xitems);
    D.n_xitems = B.get<int64_t>(1);
    D.status = B.get<int32_t>(1);
    t->queue = B.get<int32_t>(4);
    t->gs = B.get<double>(3 * nn);
    t->d_inter = B.get<unsigned long long>(1);
    t->d_useful = B.get<unsigned long long>(1);
    t->d_maxnj = B.get<int32_t>(1);
    t->d_etot = B.get<int64_t>(1);
    t->d_wsz = B.get<int64_t>(kMaxWindows);
    if (!B.ok) {
        tp_tree_free(t);
        return TP_ERR_OOM;
    }
    D.box = dbox;
    D.box_off = dboff;
    cudaMemcpyAsync(dbox, hb.data(), sizeof(BoxPrm) * nbox, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dboff, box_offsets, sizeof(int64_t) * (nbox + 1), cudaMemcpyHostToDevice, s);
    if (!alloc_nodes(t, n / 2 + 64 * (int64_t)nbox + 64)) {
        tp_tree_free(t);
        return TP_ERR_OOM;
    }
    tp_status e = run_build(t, pos, mass, s, true);
    if (e == TP_OK) e = cuda_status(cudaGetLastError());
    if (e != TP_OK) {
        tp_tree_free(t);
        return e;
    }
    *out = t;
    return TP_OK;
}

tp_status tp_build_tree(const double *pos, const double *mass, int64_t n, const tp_params *p,
                        void *stream, tp_tree **out)
{
    if (!p || n < 0) return TP_ERR_INVALID_ARG;
    const int64_t off[2] = {0, n};
    return tp_build_tree_batched(pos, mass, off, 1, p, stream, out);
}

tp_status tp_rebuild_tree(tp_tree *t, const double *pos, const double *mass, void *stream)
{
    if (!t) return TP_ERR_INVALID_ARG;
    if (t->n > 0 && !is_device_ptr(pos)) return TP_ERR_INVALID_ARG;
    if (mass && !is_device_ptr(mass)) return TP_ERR_INVALID_ARG;
    if (!t->D.gfirst || !t->D.ent || !t->D.item || !t->D.pent) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    t->last = s;
    tp_status e = run_build(t, pos, mass, s, false);
    if (e == TP_OK) e = cuda_status(cudaGetLastError());
    return e;
}

tp_status tp_refit_tree(tp_tree *t, const double *pos, const double *mass, void *stream)
{
    if (!t || t->chunked) return TP_ERR_INVALID_ARG;
    if (t->n > 0 && !is_device_ptr(pos)) return TP_ERR_INVALID_ARG;
    if (mass && !is_device_ptr(mass)) return TP_ERR_INVALID_ARG;
    if (!t->D.gfirst || !t->D.ent) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    t->last = s;
    if (t->n == 0) return TP_OK;
    tp::refit_gather(t->D, pos, mass, s);
    tp::build_moments(t->D, s);
    tp::refit_records(t->D, s);
    return cuda_status(cudaGetLastError());
}

tp_status tp_short_range_force(tp_tree *t, void *acc, void *stream)
{
    NvtxRange range("force calculation");
    if (!t || (t->n > 0 && !is_device_ptr(acc))) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    t->last = s;
    if (t->n == 0) return TP_OK;
    if (t->chunked) {
        const bool f32 = t->precision == TP_FP32;
        cudaMemsetAsync(acc, 0, (f32 ? sizeof(float) : sizeof(double)) * 3 * (size_t)t->n, s);
        t->kf_rec = false;
        tp_status e = for_each_window(t, s, [&](TreeDev &V) {
            if (f32)
                tp::pair_forward_f32(V, (float *)acc, t->queue, t->order, V.cap_groups, s, nullptr, nullptr,
                                     t->fwd_particles);
            else
                tp::pair_forward_f64(V, (double *)acc, V.cap_groups, s);
        });
        if (e != TP_OK) return e;
        return cuda_status(cudaGetLastError());
    }
    if (t->precision == TP_FP32) {
        cudaMemsetAsync(acc, 0, sizeof(float) * 3 * (size_t)t->n, s);
        tp::pair_forward_f32(t->D, (float *)acc, t->queue, t->order, t->D.cap_groups, s,
                             t->ktiming ? t->kev[0] : nullptr, t->ktiming ? t->kev[1] : nullptr, t->fwd_particles);
        t->kf_rec = t->ktiming;
    } else {
        cudaMemsetAsync(acc, 0, sizeof(double) * 3 * (size_t)t->n, s);
        tp::pair_forward_f64(t->D, (double *)acc, t->D.cap_groups, s);
    }
    return cuda_status(cudaGetLastError());
}

tp_status tp_short_range_vjp(tp_tree *t, const void *cot, double *grad, void *stream)
{
    NvtxRange range("force calculation (adjoint)");
    if (!t) return TP_ERR_INVALID_ARG;
    if (t->n > 0 && (!is_device_ptr(cot) || !is_device_ptr(grad))) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    t->last = s;
    if (t->n == 0) return TP_OK;
    if (t->chunked) {
        const bool f32 = t->precision == TP_FP32;
        t->kv_rec = false;
        tp::vjp_begin(t->D, t->gs, t->ncot, s);
        tp_status e = for_each_window(t, s, [&](TreeDev &V) {
            if (f32)
                tp::vjp_pairs_f32(V, (const float *)cot, t->gs, t->ncot, t->queue, t->order, V.cap_groups, s,
                                  nullptr, nullptr, t->adj_entries);
            else
                tp::vjp_pairs_f64(V, (const double *)cot, t->gs, t->ncot, t->queue, t->order, V.cap_groups, s);
        });
        if (e != TP_OK) return e;
        tp::vjp_end(t->D, grad, t->gs, t->ncot, leaf_scratch(t), s);
        return cuda_status(cudaGetLastError());
    }
    if (t->precision == TP_FP32)
    {
        tp::vjp_f32(t->D, (const float *)cot, grad, t->gs, t->ncot, leaf_scratch(t), t->queue, t->order,
                    t->D.cap_groups, s, t->ktiming ? t->kev[2] : nullptr, t->ktiming ? t->kev[3] : nullptr,
                    t->adj_entries);
        t->kv_rec = t->ktiming && t->D.cap_groups > 0;
    }
    else
        tp::vjp_f64(t->D, (const double *)cot, grad, t->gs, t->ncot, leaf_scratch(t), t->queue, t->order,
                    t->D.cap_groups, s);
    return cuda_status(cudaGetLastError());
}

tp_status tp_short_range_force_vjp(tp_tree *t, void *acc, const void *cot, double *grad, void *stream)
{
    NvtxRange range("force calculation (forward and adjoint)");
    if (!t) return TP_ERR_INVALID_ARG;
    if (t->n > 0 && (!is_device_ptr(acc) || !is_device_ptr(cot) || !is_device_ptr(grad)))
        return TP_ERR_INVALID_ARG;
    if (t->precision != TP_FP32) {           // the plain FP64 path: the two calls in turn
        tp_status e = tp_short_range_force(t, acc, stream);
        return e == TP_OK ? tp_short_range_vjp(t, cot, grad, stream) : e;
    }
    cudaStream_t s = (cudaStream_t)stream;
    t->last = s;
    if (t->n == 0) return TP_OK;
    cudaMemsetAsync(acc, 0, sizeof(float) * 3 * (size_t)t->n, s);
    tp::vjp_begin(t->D, t->gs, t->ncot, s);
    t->kf_rec = false;
    if (t->chunked) {
        t->kv_rec = false;
        tp_status e = for_each_window(t, s, [&](TreeDev &V) {
            tp::force_vjp_pairs_f32(V, (float *)acc, (const float *)cot, t->gs, t->ncot, t->queue, t->order,
                                    V.cap_groups, s, nullptr, nullptr, t->adj_entries);
        });
        if (e != TP_OK) return e;
    } else {
        tp::force_vjp_pairs_f32(t->D, (float *)acc, (const float *)cot, t->gs, t->ncot, t->queue, t->order,
                                t->D.cap_groups, s, t->ktiming ? t->kev[2] : nullptr,
                                t->ktiming ? t->kev[3] : nullptr, t->adj_entries);
        t->kv_rec = t->ktiming && t->D.cap_groups > 0;
    }
    tp::vjp_end(t->D, grad, t->gs, t->ncot, leaf_scratch(t), s);
    return cuda_status(cudaGetLastError());
}

tp_status tp_tree_status(tp_tree *t)
{
    if (!t) return TP_ERR_INVALID_ARG;
    tp_status e = cuda_status(cudaStreamSynchronize(t->last));
    if (e != TP_OK) return e;
    int32_t st = 0;
    e = cuda_status(cudaMemcpy(&st, t->D.status, sizeof(st), cudaMemcpyDeviceToHost));
    if (e != TP_OK) return e;
    return (tp_status)st;
}

// Statistics; the useful-pair count (a pass over every pair of the lists)
// only when asked for: the parity exports read the sizes alone.
static tp_status tree_stats(tp_tree *t, tp_stats *out, bool count)
{
    if (!t || !out) return TP_ERR_INVALID_ARG;
    cudaStream_t s = t->last;
    const bool whole = !t->chunked && t->D.gfirst;
    if (!t->chunked) {
        cudaMemsetAsync(t->d_inter, 0, sizeof(unsigned long long), s);
        cudaMemsetAsync(t->d_maxnj, 0, sizeof(int32_t), s);
        if (t->D.gfirst) tp::list_stats(t->D, t->d_inter, t->d_maxnj, s);
    }
    if (count && whole) {
        cudaMemsetAsync(t->d_useful, 0, sizeof(unsigned long long), s);
        tp::count_useful(t->D, t->d_useful, s);
    }
    unsigned long long inter = 0, amb = 0, useful = 0;
    int32_t mx = 0;
    int64_t nn = 0, ng = 0, ne = 0;
    cudaMemcpyAsync(&inter, t->d_inter, sizeof(inter), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&amb, t->D.n_ambig, sizeof(amb), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&mx, t->d_maxnj, sizeof(mx), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&nn, t->D.n_nodes, sizeof(nn), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&ng, t->D.n_groups, sizeof(ng), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&ne, t->chunked ? t->d_etot : t->D.n_entries, sizeof(ne), cudaMemcpyDeviceToHost, s);
    if (count && whole) cudaMemcpyAsync(&useful, t->d_useful, sizeof(useful), cudaMemcpyDeviceToHost, s);
    tp_status e = cuda_status(cudaStreamSynchronize(s));
    if (e != TP_OK) return e;
    if (t->n == 0) nn = ng = ne = 0;
    out->n = t->n;
    out->n_nodes = nn;
    out->n_groups = ng;
    out->n_entries = ne;
    out->n_interactions = (int64_t)inter;
    out->n_useful = t->chunked ? -1 : (int64_t)useful;
    out->n_ambiguous = (int64_t)amb;
    out->mean_ni = ng ? (double)t->n / (double)ng : 0.0;
    out->mean_nj = ng ? (double)ne / (double)ng : 0.0;
    out->max_nj = mx;
    out->nbox = t->nbox;
    out->n_windows = t->chunked ? (int64_t)t->win_count.size() : 1;
    return TP_OK;
}

tp_status tp_tree_stats(tp_tree *t, tp_stats *out) { return tree_stats(t, out, true); }

tp_status tp_export_keys(tp_tree *t, uint64_t *keys, int64_t *perm)
{
    if (!t || (t->n > 0 && (!keys || !perm))) return TP_ERR_INVALID_ARG;
    if (t->n == 0) return TP_OK;
    cudaStreamSynchronize(t->last);
    std::vector<uint32_t> p((size_t)t->n);
    tp_status e = cuda_status(cudaMemcpy(keys, t->D.key, sizeof(uint64_t) * t->n, cudaMemcpyDeviceToHost));
    if (e == TP_OK) e = cuda_status(cudaMemcpy(p.data(), t->D.perm, sizeof(uint32_t) * t->n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < t->n; i++) perm[i] = p[i];
    return e;
}

tp_status tp_export_nodes(tp_tree *t, int64_t *ints, double *dbl)
{
    if (!t) return TP_ERR_INVALID_ARG;
    tp_stats st;
    tp_status e = tree_stats(t, &st, false);
    if (e != TP_OK) return e;
    const int64_t nn = st.n_nodes;
    if (nn > 0 && (!ints || !dbl)) return TP_ERR_INVALID_ARG;
    const TreeDev &D = t->D;
    auto lv = fetch(D.level, nn);
    auto f = fetch(D.first, nn), c = fetch(D.count, nn), ch = fetch(D.child, nn), nc = fetch(D.nchild, nn),
         pa = fetch(D.parent, nn), bx = fetch(D.nbx, nn);
    const double *arrs[16] = {D.M, D.comx, D.comy, D.comz, D.lox, D.loy, D.loz, D.hix,
                              D.hiy, D.hiz, D.cenx, D.ceny, D.cenz, D.hfx, D.hfy, D.hfz};
    for (int k = 0; k < 16; k++) {
        auto v = fetch(arrs[k], nn);
        for (int64_t i = 0; i < nn; i++) dbl[16 * i + k] = v[i];
    }
    for (int64_t i = 0; i < nn; i++) {
        int64_t *a = ints + 7 * i;
        a[0] = lv[i]; a[1] = f[i]; a[2] = c[i]; a[3] = nc[i] ? ch[i] : -1; a[4] = nc[i];
        a[5] = pa[i]; a[6] = bx[i];
    }
    return cuda_status(cudaGetLastError());
}

tp_status tp_export_groups(tp_tree *t, int64_t *ints, double *dbl)
{
    if (!t) return TP_ERR_INVALID_ARG;
    tp_stats st;
    tp_status e = tree_stats(t, &st, false);
    if (e != TP_OK) return e;
    const int64_t ng = st.n_groups;
    if (ng > 0 && (!ints || !dbl)) return TP_ERR_INVALID_ARG;
    const TreeDev &D = t->D;
    auto f = fetch(D.gfirst, ng), c = fetch(D.gcount, ng), b = fetch(D.gbox, ng);
    const double *arrs[6] = {D.gcx, D.gcy, D.gcz, D.ghx, D.ghy, D.ghz};
    for (int k = 0; k < 6; k++) {
        auto v = fetch(arrs[k], ng);
        for (int64_t g = 0; g < ng; g++) dbl[6 * g + k] = v[g];
    }
    for (int64_t g = 0; g < ng; g++) {
        ints[3 * g] = f[g]; ints[3 * g + 1] = c[g]; ints[3 * g + 2] = b[g];
    }
    return cuda_status(cudaGetLastError());
}

tp_status tp_export_lists(tp_tree *t, int64_t *offsets, int32_t *entries)
{
    if (!t || !offsets || t->chunked) return TP_ERR_INVALID_ARG;
    tp_stats st;
    tp_status e = tree_stats(t, &st, false);
    if (e != TP_OK) return e;
    if (st.n_entries > 0 && !entries) return TP_ERR_INVALID_ARG;
    offsets[0] = 0;
    if (st.n_groups > 0) {
        e = cuda_status(cudaMemcpy(offsets, t->D.loff, sizeof(int64_t) * st.n_groups, cudaMemcpyDeviceToHost));
        offsets[st.n_groups] = st.n_entries;
    }
    if (e == TP_OK && st.n_entries > 0)
        e = cuda_status(cudaMemcpy(entries, t->D.ent, sizeof(int32_t) * st.n_entries, cudaMemcpyDeviceToHost));
    return e;
}

tp_status tp_tree_set_walk_budget(tp_tree *t, int64_t budget)
{
    if (!t || budget < 0) return TP_ERR_INVALID_ARG;
    t->D.walk_budget = budget;
    return TP_OK;
}

tp_status tp_tree_set_tile(tp_tree *t, int32_t fwd_particles, int32_t adj_entries)
{
    if (!t || (fwd_particles != 1 && fwd_particles != 2 && fwd_particles != 4) ||
        (adj_entries != 2 && adj_entries != 4 && adj_entries != 8))
        return TP_ERR_INVALID_ARG;
    t->fwd_particles = fwd_particles;
    t->adj_entries = adj_entries;
    return TP_OK;
}

tp_status tp_tree_set_kernel_timing(tp_tree *t, int32_t enable)
{
    if (!t) return TP_ERR_INVALID_ARG;
    if (enable && !t->kev[0]) {
        for (auto &e : t->kev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return TP_ERR_CUDA;
            }
    }
    t->ktiming = enable != 0;
    t->kf_rec = t->kv_rec = false;
    return TP_OK;
}

tp_status tp_tree_kernel_ms(tp_tree *t, double *force_ms, double *vjp_ms)
{
    if (!t || !force_ms || !vjp_ms) return TP_ERR_INVALID_ARG;
    *force_ms = -1.0;
    *vjp_ms = -1.0;
    float ms = 0.f;
    if (t->kf_rec) {
        tp_status e = cuda_status(cudaEventSynchronize(t->kev[1]));
        if (e == TP_OK) e = cuda_status(cudaEventElapsedTime(&ms, t->kev[0], t->kev[1]));
        if (e != TP_OK) return e;
        *force_ms = ms;
    }
    if (t->kv_rec) {
        tp_status e = cuda_status(cudaEventSynchronize(t->kev[3]));
        if (e == TP_OK) e = cuda_status(cudaEventElapsedTime(&ms, t->kev[2], t->kev[3]));
        if (e != TP_OK) return e;
        *vjp_ms = ms;
    }
    return TP_OK;
}

tp_status tp_tree_free(tp_tree *t)
{
    if (!t) return TP_OK;
    if (t->last) cudaStreamSynchronize(t->last);
    else cudaDeviceSynchronize();
    if (t->side) cudaStreamSynchronize(t->side);   // a build that stopped early may not have joined it
    for (auto &e : t->kev)
        if (e) cudaEventDestroy(e);
    for (auto &e : t->sev)
        if (e) cudaEventDestroy(e);
    if (t->side) cudaStreamDestroy(t->side);
    t->lists.release();
    t->pad.release();
    t->items.release();
    t->groups.release();
    t->nodes.release();
    t->base.release();
    delete t;
    cudaGetLastError();
    return TP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Leapfrog helpers and the FMA peak microbenchmark
// ---------------------------------------------------------------------------
__global__ void k_axpy(double *y, const void *x, int x_is_f32, double a, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += a * (x_is_f32 ? (double)((const float *)x)[i] : ((const double *)x)[i]);
}

__global__ void k_scale(void *out, int out_is_f32, const double *x, double a, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = a * x[i];
        if (out_is_f32) ((float *)out)[i] = (float)v;
        else ((double *)out)[i] = v;
    }
}

constexpr int kPeakChains = 8;
constexpr int kPeakIters = 4096;

__global__ void k_peak_f32(float *sink, float seed)
{
    float a[kPeakChains];
    const float m = 0.999999f, c = 1e-7f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) a[k] = seed + threadIdx.x * 1e-3f + k;
    for (int it = 0; it < kPeakIters; it++)
#pragma unroll
        for (int k = 0; k < kPeakChains; k++) a[k] = fmaf(a[k], m, c);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += a[k];
    if (s == 12345.678f) sink[0] = s;
}

__global__ void k_peak_f32x2(float *sink, float seed)
{
    unsigned long long a[kPeakChains];
    float2 mm = make_float2(0.999999f, 0.999999f), cc = make_float2(1e-7f, 1e-7f);
    const unsigned long long m = *reinterpret_cast<unsigned long long *>(&mm);
    const unsigned long long c = *reinterpret_cast<unsigned long long *>(&cc);
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) {
        float2 v = make_float2(seed + threadIdx.x * 1e-3f + k, seed + k * 0.5f);
        a[k] = *reinterpret_cast<unsigned long long *>(&v);
    }
    for (int it = 0; it < kPeakIters; it++)
#pragma unroll
        for (int k = 0; k < kPeakChains; k++)
            asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(m), "l"(c));
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) {
        float2 v = *reinterpret_cast<float2 *>(&a[k]);
        s += v.x + v.y;
    }
    if (s == 12345.678f) sink[0] = s;
}

__global__ void k_peak_f64(double *sink, double seed)
{
    double a[kPeakChains];
    const double m = 0.999999, c = 1e-7;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) a[k] = seed + threadIdx.x * 1e-3 + k;
    for (int it = 0; it < kPeakIters / 16; it++)
#pragma unroll
        for (int k = 0; k < kPeakChains; k++) a[k] = fma(a[k], m, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) s += a[k];
    if (s == 12345.678) sink[0] = s;
}

extern "C" {

tp_status tp_axpy(double *y, const void *x, int32_t x_is_f32, double a, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!is_device_ptr(y) || !is_device_ptr(x)))) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    TP_LAUNCH(k_axpy, tp::grid_for(n, 256), 256, 0, (cudaStream_t)stream, y, x, x_is_f32, a, n);
    return cuda_status(cudaGetLastError());
}

tp_status tp_scale(void *out, int32_t out_is_f32, const double *x, double a, int64_t n, void *stream)
{
    if (n < 0 || (n > 0 && (!is_device_ptr(out) || !is_device_ptr(x)))) return TP_ERR_INVALID_ARG;
    if (n == 0) return TP_OK;
    TP_LAUNCH(k_scale, tp::grid_for(n, 256), 256, 0, (cudaStream_t)stream, out, out_is_f32, x, a, n);
    return cuda_status(cudaGetLastError());
}

tp_status tp_measure_peak(int32_t kind, double *flops, void *stream)
{
    if (!flops || kind < 0 || kind > 2) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    void *sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return TP_ERR_OOM;
    const int threads = 256;
    const int blocks = tp::num_sms() * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double per_thread = 0.0;
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(a, s);
        if (kind == 0) {
            TP_LAUNCH(k_peak_f32, blocks, threads, 0, s, (float *)sink, 1.0f);
            per_thread = 2.0 * kPeakChains * kPeakIters;
        } else if (kind == 1) {
            TP_LAUNCH(k_peak_f32x2, blocks, threads, 0, s, (float *)sink, 1.0f);
            per_thread = 4.0 * kPeakChains * kPeakIters;
        } else {
            TP_LAUNCH(k_peak_f64, blocks, threads, 0, s, (double *)sink, 1.0);
            per_thread = 2.0 * kPeakChains * (kPeakIters / 16);
        }
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    *flops = per_thread * threads * (double)blocks / (best * 1e-3);
    return cuda_status(cudaGetLastError());
}

int64_t tp_launch_count(void) { return (int64_t)g_launches.load(); }

const char *tp_status_string(tp_status s)
{
    switch (s) {
    case TP_OK: return "ok";
    case TP_ERR_INVALID_ARG: return "invalid argument";
    case TP_ERR_CUDA: return "CUDA runtime error";
    case TP_ERR_OOM: return "device out of memory";
    case TP_ERR_LIST_OVERFLOW: return "capacity overflow";
    case TP_ERR_TIMEOUT: return "device wait timed out";
    case TP_ERR_NONFINITE: return "non-finite position";
    case TP_ERR_NO_DEVICE: return "no CUDA device";
    }
    return "unknown status";
}

}  // extern "C"
