// tg_host.hpp -- host-side handle and helpers of libtg (not part of the ABI).
#pragma once

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "tg.h"
#include "tg_internal.cuh"

namespace tg {

// Internal error carrying a tg_status; caught at every extern "C" entry.
struct Error {
    tg_status status;
    const char *what;
    bool from_cuda = false;     // message already recorded by throw_cuda
};

// Text of the calling thread's last failed entry (tg_last_error).
inline thread_local char tl_last_error[256] = "";

inline void throw_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    (void)cudaGetLastError();   // clear the sticky-free error state
    std::snprintf(tl_last_error, sizeof tl_last_error, "%s: %s", what, cudaGetErrorString(e));
    throw Error{e == cudaErrorMemoryAllocation ? TG_ERR_OOM : TG_ERR_CUDA, what, true};
}

// Raises (never lowers) a kernel's dynamic shared-memory limit.  The limit
// is a process-wide attribute of the function, so handles counted
// concurrently on several host threads must not shrink it under one another.
// Defined in tg_count.cu.
void raise_smem_limit(const void *func, size_t bytes);

// Largest light_anchor_max_wedges whose per-warp hashes of k_wedge_light fit
// one CTA's shared memory for L types.  Defined in tg_count.cu.
int light_anchor_limit(int L);

#define TG_CK(call) ::tg::throw_cuda((call), #call)

// Stream-ordered memory pool of the current device, owned by the library
// (release threshold kept at its maximum, so freed blocks are reused instead
// of returned to the CUDA driver).  Defined in tg_build.cu.
cudaMemPool_t device_pool();

// Device buffer owned by a handle; freed by release() or the destructor.
// With an owner stream (the handle's stream) it is allocated and freed
// stream-ordered from the library pool, so no call synchronises the device;
// without one it falls back to cudaMalloc / cudaFree.
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    const cudaStream_t *owner = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void alloc(size_t b) {
        release();
        if (b == 0) b = 16;
        if (owner) TG_CK(cudaMallocFromPoolAsync(&p, b, device_pool(), *owner));
        else TG_CK(cudaMalloc(&p, b));
        bytes = b;
    }
    void release() {
        if (p) {
            if (owner) cudaFreeAsync(p, *owner);
            else cudaFree(p);
        }
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Temporary device buffer of one call, stream-ordered on `st`, from the
// same library pool (which keeps freed blocks mapped for the life of the
// process instead of returning them to the CUDA driver at synchronisations).
struct TBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    TBuf(size_t b, cudaStream_t st) : s(st) {
        if (b == 0) b = 16;
        TG_CK(cudaMallocFromPoolAsync(&p, b, device_pool(), s));
    }
    TBuf(const TBuf &) = delete;
    TBuf &operator=(const TBuf &) = delete;
    ~TBuf() { if (p) cudaFreeAsync(p, s); }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

inline bool is_device_pointer(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Layout of the position-aware counts (Sec. 5): per-edge blocks O1..O12
// and the classes of each global block (tg_pa.cu).
struct PaLayout {
    int32_t L = 0, S = 0;               // types, per-edge slots
    int64_t G = 0;                      // classes per graph
    int32_t off[13] = {0};              // first slot of blocks O1..O12 (index 1..12)
    int64_t bsize[9] = {0};             // classes of each global block
    int64_t boff[10] = {0};             // first class of each global block; boff[9] = G
};

struct Graph {
    int device = 0;
    cudaStream_t stream = nullptr;      // stream of the last call
    int32_t ngraphs = 1, L = 1;
    int64_t n = 0, nnz = 0, m = 0;
    int64_t max_graph_nodes = 0;
    int64_t max_degree = 0;
    std::vector<int64_t> h_node_off, h_edge_off, h_slot_off;
    // chunks of whole graphs counted one after another (bounds the 4-cycle array)
    struct Chunk { int32_t g0, g1; int64_t n0, n1, s0, s1, e0, e1, t0, t1; };
    std::vector<Chunk> chunks;
    int64_t a_stride = 0, a_base = 0;
    tg_options opt;

    // graph (built once)
    DBuf node_off, edge_off, rp, adj, toff, pivot, nplus, ty, old_of, slot_eid, e_lo, e_hi, e_slot_lo, e_slot_hi, delta;
    DBuf plus_off, plus_adj;
    // work lists
    DBuf anchors_light, anchors_heavy, edges_light, edges_heavy;
    int64_t n_anchors_light = 0, n_anchors_heavy = 0, n_edges_light = 0, n_edges_heavy = 0;
    int64_t n_heavy_dense = 0;          // leading heavy anchors with more than kHeavyFit wedges
    // hub anchors (ascending id) and their wedge items: one item per
    // (hub, lower-priority neighbour v, type of w) with at least one wedge
    DBuf hubs, hub_base, item_woff, item_rec;
    int64_t n_hubs = 0, n_items = 0;
    std::vector<int32_t> h_hub_id;      // hub node ids
    std::vector<int64_t> h_hub_wedges;  // wedges of each hub
    std::vector<int64_t> h_hub_item;    // first item of each hub (n_hubs + 1)
    std::vector<int64_t> h_hub_woff;    // first wedge of each hub (n_hubs + 1)
    bool hubs_ready = false;
    // persistent hub pass (tg_count.cu): per chunk, its ticket queue; the
    // table buffers shared by all chunks
    struct HubPlan {
        DBuf segs, groups, ntick, ctr;
        std::vector<HubGroup> h_groups;     // host copies (kept while the uploads may be in flight)
        std::vector<HubSegment> h_segs;
        std::vector<int64_t> h_ntick;       // tickets per (group, kind)
        int64_t n_tickets = 0, n_groups = 0, n_segs = 0;
    };
    std::vector<std::unique_ptr<HubPlan>> hub_plans;
    DBuf hub_tables;
    // directed counts (tg_directed.cu): slot signs, typed out-degrees, class tables
    DBuf dsign, doutdeg, dcls, darcs, dgacc;
    int64_t d_global = 0;
    bool directed = false;
    // edge-typed counts (tg_edge_typed.cu): edge type per slot, per-node
    // neighbour counts by (node type, edge type), the totals' accumulator
    DBuf etype, etdeg, etgacc;
    int32_t et_X = 0;
    int64_t et_global = 0;
    bool edge_typed = false;
    int64_t hub_stride = 0, hub_buf_words = 0;  // words per hub table, per buffer
    bool hub_packed = false;                    // two 16-bit counters per word
    // counting state
    DBuf C, tau, A, tables, gacc, status, tiles_full, stage_pe, stage_gl;
    DBuf tcount, toffs, tlist, tsum, kmat, big_list, big_count, scan_tmp, set_scratch;
    DBuf work;                          // [kWorkSlots] work counters (tg_set_work_counting)
    bool work_on = false;
    int64_t set_stride = 1;
    int32_t big_blocks = 1;
    int64_t n_tiles_full = 0, max_chunk_edges = 0, tlist_cap = 0;
    size_t scan_tmp_bytes = 0;
    std::vector<int64_t> chunk_t;       // triangle-node entries per chunk (graph invariant)
    int64_t e_base = 0;
    int64_t table_stride = 0;
    int32_t n_tables = 0;
    int32_t prepared_k = 0;             // 0: nothing, 3: C and tau, 4: C, tau and A
    int64_t last_launches = 0;
    // per-kernel event timing (tg_set_timing)
    bool timing = false;
    struct TimerRec { const char *name; cudaEvent_t a, b; };
    std::vector<TimerRec> timer_pending;
    std::vector<cudaEvent_t> event_pool;
    std::vector<std::pair<const char *, std::pair<double, int64_t>>> timer_totals;
    // position-aware counting (Sec. 5): slot -> class table, raw class sums
    DBuf pa_cls, pa_gacc;
    PaLayout pa;
    bool pa_active = false;             // the per-edge epilogue writes position-aware rows
    // CUDA graph of the last batched count
    cudaGraphExec_t batch_exec = nullptr;
    int32_t batch_k = 0;
    const void *batch_pe = nullptr, *batch_gl = nullptr;
    cudaStream_t batch_stream = nullptr;

    GraphView view() const {
        GraphView v;
        v.ngraphs = ngraphs; v.L = L; v.n = n; v.nnz = nnz; v.m = m;
        v.isect_modes = opt.isect_modes;
        v.node_off = node_off.as<int64_t>();
        v.edge_off = edge_off.as<int64_t>();
        v.rp = rp.as<int64_t>();
        v.adj = adj.as<int32_t>();
        v.toff = toff.as<int32_t>();
        v.pivot = pivot.as<int32_t>();
        v.nplus = nplus.as<int32_t>();
        v.ty = ty.as<uint8_t>();
        v.slot_eid = slot_eid.as<int32_t>();
        v.e_lo = e_lo.as<int32_t>();
        v.e_hi = e_hi.as<int32_t>();
        v.e_slot_lo = e_slot_lo.as<int64_t>();
        v.e_slot_hi = e_slot_hi.as<int64_t>();
        v.delta = delta.as<int64_t>();
        v.plus_off = plus_off.as<int64_t>();
        v.plus_adj = plus_adj.as<int32_t>();
        return v;
    }
    CountView cview() const {
        CountView c;
        c.C = C.as<uint32_t>();
        c.tau = tau.as<int64_t>();
        c.A = A.as<uint32_t>();
        c.a_base = a_base;
        c.a_stride = a_stride;
        c.e_base = e_base;
        c.toffs = toffs.as<int64_t>();
        c.tlist = tlist.as<int32_t>();
        c.tsum = tsum.as<unsigned long long>();
        c.kmat = kmat.as<unsigned long long>();
        c.tables = tables.as<uint32_t>();
        c.table_stride = table_stride;
        c.gacc = gacc.as<unsigned long long>();
        c.status = status.as<uint32_t>();
        c.work = work_on ? work.as<unsigned long long>() : nullptr;
        return c;
    }
    Graph() {
        for (DBuf *b : buffers()) b->owner = &stream;
    }
    std::vector<DBuf *> buffers() {
        std::vector<DBuf *> v;
        for (const DBuf *b : cbuffers()) v.push_back(const_cast<DBuf *>(b));
        return v;
    }
    std::vector<const DBuf *> cbuffers() const {
        return {&node_off, &edge_off, &rp, &adj, &toff, &pivot, &nplus, &ty, &old_of, &slot_eid, &e_lo, &e_hi,
                             &e_slot_lo, &e_slot_hi, &delta, &anchors_light, &anchors_heavy, &edges_light,
                             &edges_heavy, &C, &tau, &A, &tables, &gacc, &status, &tiles_full, &stage_pe,
                             &stage_gl, &tcount, &toffs, &tlist, &tsum, &kmat, &big_list, &big_count, &scan_tmp,
                             &set_scratch, &work, &hub_tables, &dsign, &doutdeg, &dcls, &darcs, &dgacc, &etype, &etdeg, &etgacc, &plus_off, &plus_adj, &hubs, &hub_base, &item_woff, &item_rec,
                &pa_cls, &pa_gacc};
    }
    int64_t device_bytes() const {
        int64_t s = 0;
        for (const DBuf *b : cbuffers()) s += (int64_t)b->bytes;
        return s;
    }
    ~Graph() {
        if (batch_exec) cudaGraphExecDestroy(batch_exec);
        for (auto &r : timer_pending) { event_pool.push_back(r.a); event_pool.push_back(r.b); }
        for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
    }
    cudaEvent_t take_event() {
        if (!event_pool.empty()) { cudaEvent_t e = event_pool.back(); event_pool.pop_back(); return e; }
        cudaEvent_t e;
        TG_CK(cudaEventCreate(&e));
        return e;
    }
};

// Brackets one kernel launch with events when timing is on and the stream
// is not being captured.
struct KernelTimer {
    Graph &G;
    cudaStream_t s;
    const char *name;
    cudaEvent_t a = nullptr, b = nullptr;
    KernelTimer(Graph &g, cudaStream_t st, const char *nm) : G(g), s(st), name(nm) {
        if (!G.timing) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
        a = G.take_event();
        b = G.take_event();
        TG_CK(cudaEventRecord(a, s));
    }
    ~KernelTimer() {
        if (!a) return;
        if (cudaEventRecord(b, s) == cudaSuccess) G.timer_pending.push_back(Graph::TimerRec{name, a, b});
    }
};

inline void fill_defaults(tg_options *o) {
    std::memset(o, 0, sizeof(*o));
    o->light_edge_max_degree = 256;
    o->light_anchor_max_wedges = 64;
    o->anchor_table_budget_mb = 12288;
    o->ctas_per_sm = 3;
    o->cycle_budget_mb = 16384;
    o->hub_min_wedges = 1 << 14;
    o->hub_l2_mb = 192;
}

// number of SMs of the current device
int sm_count();

// build entry (tg_build.cu)
void build_graph(Graph &G, int32_t ngraphs, const int64_t *node_off_host, int64_t n, int64_t nnz,
                 const int64_t *row_ptr, const int32_t *col, const uint8_t *types, int32_t L,
                 const tg_options &opt, cudaStream_t s);

// count entries (tg_count.cu)
void prepare_counting(Graph &G, int k, cudaStream_t s);
void prepare_edges(Graph &G, int k, cudaStream_t s);
void prepare_capture(Graph &G, int k, cudaStream_t s);
// Runs the counting stages for edges [e_begin, e_end) into per_edge_out
// (row 0 = e_begin) and the raw sums gacc.  full: the whole graph, every
// stage recomputed (no cached state).  Returns the kernel launches.
int64_t run_count(Graph &G, int k, int64_t e_begin, int64_t e_end, uint32_t *per_edge_out,
                  unsigned long long *gacc, bool full, cudaStream_t s);
int64_t launch_finalize(Graph &G, int k, int64_t *global_out, cudaStream_t s);
// Position-aware typed graphlets (tg_pa.cu; epilogue in tg_count.cu).
PaLayout pa_layout(int L);
bool pa_labelling(int L, int block, int64_t rank, int32_t *labelling);
std::vector<int32_t> pa_class_table(const PaLayout &Y);
void prepare_position_aware(Graph &G, cudaStream_t s);
void prepare_epi4_pa(Graph &G);
int64_t launch_finalize_pa(Graph &G, int64_t *global_out, cudaStream_t s);
// Typed-graphlet weighted graph (tg_weights.cu).
void launch_weights(Graph &G, int k, const uint32_t *rows, int block, int64_t rank, int64_t *weights,
                    int64_t *degree, cudaStream_t s);
// Directed typed 3-node graphlets (tg_directed.cu).
int64_t directed_classes(int L);
bool directed_class_code(int L, int64_t rank, int32_t *types3, int32_t *arcs3);
void symmetrize_arcs(int64_t n, int64_t na, const int64_t *orp, const int32_t *ocol, int64_t *srp, int32_t *scol,
                     int32_t *src, cudaStream_t s);
void prepare_directed(Graph &G, int64_t na, const int32_t *src, const int32_t *ocol, cudaStream_t s);
int64_t run_directed3(Graph &G, uint32_t *per_edge_out, int64_t *global_out, cudaStream_t s);
// Edge-typed 3-node graphlets (tg_edge_typed.cu).
int64_t edge_typed_global_slots(int L, int X);
void prepare_edge_typed(Graph &G, int X, const int64_t *row_ptr, const int32_t *col, const uint8_t *edge_types,
                        cudaStream_t s);
int64_t run_edge_typed3(Graph &G, uint32_t *per_edge_out, int64_t *global_out, cudaStream_t s);
// Sparse per-edge counts (tg_sparse.cu): returns the number of nonzero
// pairs; writes them only while they fit `cap` (fits = false otherwise).
int64_t count_sparse(Graph &G, int k, int64_t *row_off, uint16_t *slot, uint32_t *value, int64_t cap, bool &fits,
                     cudaStream_t s);

}  // namespace tg

struct tg_graph {
    tg::Graph g;
};
