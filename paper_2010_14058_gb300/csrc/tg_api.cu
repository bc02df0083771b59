// tg_api.cu -- the extern "C" entry points of libtg (declared in include/tg.h).
//
// Every entry catches the library's internal errors and returns a tg_status;
// nothing here traps, aborts or exits.
#include <algorithm>
#include <cstring>
#include <new>
#include <mutex>
#include <vector>

#include "tg_host.hpp"

using tg::Error;
using tg::Graph;

namespace {

template <class F>
tg_status guarded(F f) {
    try {
        f();
        return TG_OK;
    } catch (const Error &e) {
        if (!e.from_cuda)
            std::snprintf(tg::tl_last_error, sizeof tg::tl_last_error, "%s: %s", e.what ? e.what : "",
                          tg_status_string(e.status));
        return e.status;
    } catch (const std::bad_alloc &) {
        std::snprintf(tg::tl_last_error, sizeof tg::tl_last_error, "host allocation failed");
        return TG_ERR_OOM;
    } catch (...) {
        std::snprintf(tg::tl_last_error, sizeof tg::tl_last_error, "unexpected exception");
        return TG_ERR_INTERNAL;
    }
}

__global__ void k_endpoints(int64_t m, const int32_t *__restrict__ e_lo, const int32_t *__restrict__ e_hi,
                            const int32_t *__restrict__ old_of, int32_t *src, int32_t *dst) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m) return;
    int32_t a = old_of[e_lo[e]], b = old_of[e_hi[e]];
    src[e] = a < b ? a : b;
    dst[e] = a < b ? b : a;
}

void check_types(int32_t L) {
    if (L < 1 || L > TG_MAX_TYPES) throw Error{TG_ERR_TOO_MANY_TYPES, "L"};
}

void build_common(int32_t ngraphs, const int64_t *node_off, int64_t n, int64_t nnz, const int64_t *row_ptr,
                  const int32_t *col, const uint8_t *types, int32_t L, const tg_options *opt, void *stream,
                  tg_graph **out) {
    if (!out) throw Error{TG_ERR_INVALID_ARG, "out"};
    *out = nullptr;
    check_types(L);
    if (ngraphs < 1 || !node_off || n < 0 || nnz < 0 || (nnz & 1) || !row_ptr) throw Error{TG_ERR_INVALID_ARG, "sizes"};
    if ((n > 0 && !types) || (nnz > 0 && !col)) throw Error{TG_ERR_INVALID_ARG, "NULL array"};
    if (node_off[0] != 0 || node_off[ngraphs] != n) throw Error{TG_ERR_INVALID_ARG, "node_off"};
    for (int g = 0; g < ngraphs; ++g)
        if (node_off[g + 1] < node_off[g]) throw Error{TG_ERR_INVALID_ARG, "node_off"};
    if (n >= ((int64_t)1 << tg::kTypeShift) || nnz >= ((int64_t)1 << 31)) throw Error{TG_ERR_TOO_LARGE, "index width"};
    tg_options o;
    tg::fill_defaults(&o);
    if (opt) {
        if (opt->light_edge_max_degree > 0) o.light_edge_max_degree = opt->light_edge_max_degree;
        if (opt->light_anchor_max_wedges > 0) o.light_anchor_max_wedges = opt->light_anchor_max_wedges;
        if (opt->anchor_table_budget_mb > 0) o.anchor_table_budget_mb = opt->anchor_table_budget_mb;
        if (opt->ctas_per_sm > 0) o.ctas_per_sm = opt->ctas_per_sm;
        if (opt->cycle_budget_mb > 0) o.cycle_budget_mb = opt->cycle_budget_mb;
        if (opt->hub_min_wedges > 0) o.hub_min_wedges = opt->hub_min_wedges;
        if (opt->hub_l2_mb > 0) o.hub_l2_mb = opt->hub_l2_mb;
        if (opt->isect_modes > 0) o.isect_modes = opt->isect_modes & 0xff;
    }
    o.hub_min_wedges = std::max(o.hub_min_wedges, o.light_anchor_max_wedges);
    o.light_edge_max_degree = std::min(o.light_edge_max_degree, 256);     // warp T list capacity
    o.light_anchor_max_wedges = std::min({o.light_anchor_max_wedges, 2048, tg::light_anchor_limit(L)});
    o.ctas_per_sm = std::min(std::max(o.ctas_per_sm, 1), 8);
    tg_graph *h = new tg_graph();
    try {
        tg::build_graph(h->g, ngraphs, node_off, n, nnz, row_ptr, col, types, L, o, (cudaStream_t)stream);
    } catch (...) {
        cudaStreamSynchronize((cudaStream_t)stream);
        h->g.stream = nullptr;
        delete h;
        throw;
    }
    *out = h;
}

// device pointer for an output, staged through `stage` when the caller passed host memory
template <class T>
T *device_out(T *p, size_t bytes, tg::DBuf &stage, bool &staged) {
    staged = false;
    if (!p) return nullptr;
    if (tg::is_device_pointer(p)) return p;
    if (stage.bytes < bytes) stage.alloc(bytes);
    staged = true;
    return stage.as<T>();
}

}  // namespace

extern "C" {

tg_status tg_layout(int32_t L, int32_t k, tg_layout_t *out) {
    return guarded([&] {
        check_types(L);
        if ((k != 3 && k != 4) || !out) throw Error{TG_ERR_INVALID_ARG, "k"};
        tg_layout_t r;
        std::memset(&r, 0, sizeof(r));
        r.L = L;
        r.k = k;
        r.pairs = tg::npairs(L);
        r.per_edge_slots = tg::per_edge_slots(L, k);
        r.global_slots = tg::global_slots(L, k);
        r.orbit_offset[1] = 0;
        r.orbit_offset[2] = L;
        for (int o = 3; o <= 12; ++o) r.orbit_offset[o] = k == 4 ? 2 * L + (o - 3) * r.pairs : -1;
        const int edges_of[9] = {1, 2, 3, 3, 3, 4, 4, 5, 6};
        int64_t off = 0;
        for (int b = 0; b < 9; ++b) {
            int64_t sz = b == 0 ? tg::binom_small(L + 1, 2) : (b <= 2 ? tg::binom_small(L + 2, 3) : tg::binom_small(L + 3, 4));
            if (k == 3 && b > 2) sz = 0;
            r.global_block_offset[b] = off;
            r.global_block_size[b] = sz;
            r.graphlet_edges[b] = edges_of[b];
            off += sz;
        }
        *out = r;
    });
}

tg_status tg_pa_layout(int32_t L, tg_pa_layout_t *out) {
    return guarded([&] {
        check_types(L);
        if (!out) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        const tg::PaLayout Y = tg::pa_layout(L);
        tg_pa_layout_t r;
        std::memset(&r, 0, sizeof(r));
        r.L = L;
        r.per_edge_slots = Y.S;
        r.global_slots = Y.G;
        for (int o = 1; o <= 12; ++o) r.block_offset[o] = Y.off[o];
        const int edges_of[9] = {1, 2, 3, 3, 3, 4, 4, 5, 6};
        for (int b = 0; b < 9; ++b) {
            r.global_block_offset[b] = Y.boff[b];
            r.global_block_size[b] = Y.bsize[b];
            r.graphlet_edges[b] = edges_of[b];
        }
        *out = r;
    });
}

tg_status tg_pa_labelling(int32_t L, int32_t block, int64_t rank, int32_t *types_out) {
    return guarded([&] {
        check_types(L);
        if (!types_out || block < 0 || block > 8) throw Error{TG_ERR_INVALID_ARG, "block"};
        if (!tg::pa_labelling(L, block, rank, types_out)) throw Error{TG_ERR_INVALID_ARG, "rank"};
    });
}

tg_status tg_pa_slot_class(int32_t L, int32_t phi_lo, int32_t phi_hi, int64_t slot, int64_t *class_out) {
    return guarded([&] {
        check_types(L);
        if (!class_out || phi_lo < 0 || phi_lo >= L || phi_hi < 0 || phi_hi >= L)
            throw Error{TG_ERR_INVALID_ARG, "types"};
        // one table per L, built on first use and kept (a few hundred KB at most)
        static std::mutex mu;
        static std::vector<int32_t> tables[TG_MAX_TYPES + 1];
        static int32_t slots[TG_MAX_TYPES + 1];
        std::lock_guard<std::mutex> lock(mu);
        if (tables[L].empty()) {
            const tg::PaLayout Y = tg::pa_layout(L);
            tables[L] = tg::pa_class_table(Y);
            slots[L] = Y.S;
        }
        if (slot < 0 || slot > slots[L]) throw Error{TG_ERR_INVALID_ARG, "slot"};
        *class_out = tables[L][(size_t)(phi_lo * L + phi_hi) * (slots[L] + 1) + slot];
    });
}

void tg_default_options(tg_options *opt) {
    if (opt) tg::fill_defaults(opt);
}

tg_status tg_build(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col, const uint8_t *node_types,
                   int32_t L, const tg_options *opt, void *stream, tg_graph **out) {
    const int64_t off[2] = {0, n};
    return guarded([&] { build_common(1, off, n, nnz, row_ptr, col, node_types, L, opt, stream, out); });
}

tg_status tg_build_batch(int32_t ngraphs, const int64_t *node_off, int64_t n, int64_t nnz, const int64_t *row_ptr,
                         const int32_t *col, const uint8_t *node_types, int32_t L, const tg_options *opt,
                         void *stream, tg_graph **out) {
    return guarded([&] { build_common(ngraphs, node_off, n, nnz, row_ptr, col, node_types, L, opt, stream, out); });
}

tg_status tg_directed_layout(int32_t L, tg_directed_layout_t *out) {
    return guarded([&] {
        check_types(L);
        if (!out) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        tg_directed_layout_t r;
        std::memset(&r, 0, sizeof(r));
        r.L = L;
        r.per_edge_slots = 8 * (int64_t)L;
        r.classes = tg::directed_classes(L);
        r.global_slots = (int64_t)L * L + r.classes;
        *out = r;
    });
}

tg_status tg_directed_class_code(int32_t L, int64_t rank, int32_t *types3, int32_t *arcs3) {
    return guarded([&] {
        check_types(L);
        if (!types3 || !arcs3) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        if (!tg::directed_class_code(L, rank, types3, arcs3)) throw Error{TG_ERR_INVALID_ARG, "rank"};
    });
}

tg_status tg_build_directed(int64_t n, int64_t n_arcs, const int64_t *out_row_ptr, const int32_t *out_col,
                            const uint8_t *node_types, int32_t L, const tg_options *opt, void *stream, tg_graph **out) {
    return guarded([&] {
        if (!out) throw Error{TG_ERR_INVALID_ARG, "out"};
        *out = nullptr;
        check_types(L);
        if (n < 0 || n_arcs < 0 || !out_row_ptr || (n_arcs > 0 && !out_col) || (n > 0 && !node_types))
            throw Error{TG_ERR_INVALID_ARG, "sizes"};
        if (2 * n_arcs >= ((int64_t)1 << 31) || n >= ((int64_t)1 << tg::kTypeShift))
            throw Error{TG_ERR_TOO_LARGE, "index width"};
        cudaStream_t s = (cudaStream_t)stream;
        // row pointers checked on the host; arcs on the device
        std::vector<int64_t> orp((size_t)n + 1);
        const bool dev_rp = tg::is_device_pointer(out_row_ptr), dev_col = tg::is_device_pointer(out_col);
        TG_CK(cudaMemcpyAsync(orp.data(), out_row_ptr, sizeof(int64_t) * (n + 1),
                              dev_rp ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
        TG_CK(cudaStreamSynchronize(s));
        if (orp[0] != 0 || orp[(size_t)n] != n_arcs) throw Error{TG_ERR_INVALID_GRAPH, "row pointers"};
        for (int64_t v = 0; v < n; ++v)
            if (orp[(size_t)v + 1] < orp[(size_t)v]) throw Error{TG_ERR_INVALID_GRAPH, "row pointers"};
        tg::TBuf drp(sizeof(int64_t) * (n + 1), s), dcol(sizeof(int32_t) * std::max<int64_t>(n_arcs, 1), s);
        TG_CK(cudaMemcpyAsync(drp.p, orp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
        if (n_arcs > 0)
            TG_CK(cudaMemcpyAsync(dcol.p, out_col, sizeof(int32_t) * n_arcs,
                                  dev_col ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        tg::TBuf srp(sizeof(int64_t) * (n + 1), s), scol(sizeof(int32_t) * std::max<int64_t>(2 * n_arcs, 1), s),
            src(sizeof(int32_t) * std::max<int64_t>(n_arcs, 1), s);
        tg::symmetrize_arcs(n, n_arcs, drp.as<int64_t>(), dcol.as<int32_t>(), srp.as<int64_t>(), scol.as<int32_t>(),
                            src.as<int32_t>(), s);
        const int64_t off[2] = {0, n};
        tg_graph *h = nullptr;
        build_common(1, off, n, 2 * n_arcs, srp.as<int64_t>(), scol.as<int32_t>(), node_types, L, opt, stream, &h);
        try {
            tg::prepare_directed(h->g, n_arcs, src.as<int32_t>(), dcol.as<int32_t>(), s);
        } catch (...) {
            tg_free(h);
            throw;
        }
        *out = h;
    });
}

tg_status tg_count_directed3(tg_graph *gh, uint32_t *per_edge_out, int64_t *global_out, void *stream) {
    return guarded([&] {
        if (!gh || !gh->g.directed) throw Error{TG_ERR_INVALID_ARG, "not a directed handle"};
        Graph &G = gh->g;
        cudaStream_t s = (cudaStream_t)stream;
        G.stream = s;
        const size_t pe_bytes = (size_t)G.m * 8 * G.L * sizeof(uint32_t);
        const size_t gl_bytes = (size_t)G.d_global * sizeof(int64_t);
        bool pe_staged = false, gl_staged = false;
        uint32_t *pe = device_out(per_edge_out, pe_bytes, G.stage_pe, pe_staged);
        int64_t *gl = device_out(global_out, gl_bytes, G.stage_gl, gl_staged);
        G.last_launches = tg::run_directed3(G, pe, gl, s);
        if (pe_staged && pe_bytes) TG_CK(cudaMemcpyAsync(per_edge_out, pe, pe_bytes, cudaMemcpyDeviceToHost, s));
        if (gl_staged) TG_CK(cudaMemcpyAsync(global_out, gl, gl_bytes, cudaMemcpyDeviceToHost, s));
        if (pe_staged || gl_staged) TG_CK(cudaStreamSynchronize(s));
    });
}

tg_status tg_edge_typed_layout(int32_t L, int32_t X, tg_edge_typed_layout_t *out) {
    return guarded([&] {
        check_types(L);
        if (X < 1 || X > TG_MAX_EDGE_TYPES) throw Error{TG_ERR_TOO_MANY_TYPES, "edge types"};
        if (!out) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        tg_edge_typed_layout_t r;
        std::memset(&r, 0, sizeof(r));
        r.L = L;
        r.X = X;
        const int64_t P = (int64_t)X * (X + 1) / 2;
        r.per_edge_slots = (int64_t)L * X + (int64_t)L * P;
        r.triangle_offset = (int64_t)L * X;
        const int64_t c2 = (int64_t)L * (L + 1) / 2, c3 = (int64_t)L * (L + 1) * (L + 2) / 6;
        r.global_block_size[0] = c2 * X;
        r.global_block_size[1] = c3 * P;
        r.global_block_size[2] = c3 * ((int64_t)X * (X + 1) * (X + 2) / 6);
        r.global_block_offset[0] = 0;
        r.global_block_offset[1] = r.global_block_size[0];
        r.global_block_offset[2] = r.global_block_size[0] + r.global_block_size[1];
        r.global_slots = tg::edge_typed_global_slots(L, X);
        *out = r;
    });
}

tg_status tg_build_edge_typed(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                              const uint8_t *node_types, const uint8_t *edge_types, int32_t L, int32_t X,
                              const tg_options *opt, void *stream, tg_graph **out) {
    return guarded([&] {
        if (!out) throw Error{TG_ERR_INVALID_ARG, "out"};
        *out = nullptr;
        check_types(L);
        if (X < 1 || X > TG_MAX_EDGE_TYPES) throw Error{TG_ERR_TOO_MANY_TYPES, "edge types"};
        if (nnz > 0 && !edge_types) throw Error{TG_ERR_INVALID_ARG, "edge_types"};
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t off[2] = {0, n};
        tg_graph *h = nullptr;
        build_common(1, off, n, nnz, row_ptr, col, node_types, L, opt, stream, &h);
        try {
            // device copies of the caller's CSR positions and their edge types
            tg::TBuf drp(sizeof(int64_t) * (n + 1), s), dcol(sizeof(int32_t) * std::max<int64_t>(nnz, 1), s),
                dxi(std::max<int64_t>(nnz, 1), s);
            auto kind = [](const void *p) {
                return tg::is_device_pointer(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            };
            TG_CK(cudaMemcpyAsync(drp.p, row_ptr, sizeof(int64_t) * (n + 1), kind(row_ptr), s));
            if (nnz > 0) {
                TG_CK(cudaMemcpyAsync(dcol.p, col, sizeof(int32_t) * nnz, kind(col), s));
                TG_CK(cudaMemcpyAsync(dxi.p, edge_types, nnz, kind(edge_types), s));
            }
            tg::prepare_edge_typed(h->g, X, drp.as<int64_t>(), dcol.as<int32_t>(), dxi.as<uint8_t>(), s);
        } catch (...) {
            tg_free(h);
            throw;
        }
        *out = h;
    });
}

tg_status tg_count_edge_typed3(tg_graph *gh, uint32_t *per_edge_out, int64_t *global_out, void *stream) {
    return guarded([&] {
        if (!gh || !gh->g.edge_typed) throw Error{TG_ERR_INVALID_ARG, "not an edge-typed handle"};
        Graph &G = gh->g;
        cudaStream_t s = (cudaStream_t)stream;
        G.stream = s;
        const int64_t X = G.et_X, P = X * (X + 1) / 2;
        const size_t pe_bytes = (size_t)G.m * (size_t)(G.L * X + G.L * P) * sizeof(uint32_t);
        const size_t gl_bytes = (size_t)G.et_global * sizeof(int64_t);
        bool pe_staged = false, gl_staged = false;
        uint32_t *pe = device_out(per_edge_out, pe_bytes, G.stage_pe, pe_staged);
        int64_t *gl = device_out(global_out, gl_bytes, G.stage_gl, gl_staged);
        G.last_launches = tg::run_edge_typed3(G, pe, gl, s);
        if (pe_staged && pe_bytes) TG_CK(cudaMemcpyAsync(per_edge_out, pe, pe_bytes, cudaMemcpyDeviceToHost, s));
        if (gl_staged) TG_CK(cudaMemcpyAsync(global_out, gl, gl_bytes, cudaMemcpyDeviceToHost, s));
        if (pe_staged || gl_staged) TG_CK(cudaStreamSynchronize(s));
    });
}

void tg_free(tg_graph *g) {
    if (!g) return;
    cudaStreamSynchronize(g->g.stream);
    g->g.stream = nullptr;          // release on the legacy stream: the caller's may be gone later
    delete g;
}

int64_t tg_num_nodes(const tg_graph *g) { return g ? g->g.n : -1; }
int64_t tg_num_edges(const tg_graph *g) { return g ? g->g.m : -1; }
int32_t tg_num_graphs(const tg_graph *g) { return g ? g->g.ngraphs : -1; }
int32_t tg_num_types(const tg_graph *g) { return g ? g->g.L : -1; }
int64_t tg_device_bytes(const tg_graph *g) { return g ? g->g.device_bytes() : -1; }
int64_t tg_last_launch_count(const tg_graph *g) { return g ? g->g.last_launches : -1; }
int32_t tg_abi_version(void) { return TG_ABI_VERSION; }

tg_status tg_edge_endpoints(const tg_graph *gh, int32_t *src, int32_t *dst) {
    return guarded([&] {
        if (!gh || !src || !dst) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        const Graph &G = gh->g;
        cudaStream_t s = G.stream;
        const size_t bytes = sizeof(int32_t) * (size_t)std::max<int64_t>(G.m, 1);
        bool dev_s = tg::is_device_pointer(src), dev_d = tg::is_device_pointer(dst);
        tg::TBuf ts(dev_s ? 0 : bytes, s), td(dev_d ? 0 : bytes, s);
        int32_t *ps = dev_s ? src : ts.as<int32_t>(), *pd = dev_d ? dst : td.as<int32_t>();
        if (G.m > 0) {
            k_endpoints<<<(unsigned)((G.m + 255) / 256), 256, 0, s>>>(G.m, G.e_lo.as<int32_t>(), G.e_hi.as<int32_t>(),
                                                                  G.old_of.as<int32_t>(), ps, pd);
            TG_CK(cudaGetLastError());
            if (!dev_s) TG_CK(cudaMemcpyAsync(src, ps, sizeof(int32_t) * G.m, cudaMemcpyDeviceToHost, s));
            if (!dev_d) TG_CK(cudaMemcpyAsync(dst, pd, sizeof(int32_t) * G.m, cudaMemcpyDeviceToHost, s));
        }
        TG_CK(cudaStreamSynchronize(s));
    });
}

tg_status tg_edge_offsets(const tg_graph *gh, int64_t *out) {
    return guarded([&] {
        if (!gh || !out) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        std::copy(gh->g.h_edge_off.begin(), gh->g.h_edge_off.end(), out);
    });
}

tg_status tg_count(tg_graph *gh, int32_t k, uint32_t *per_edge_out, int64_t *global_out, void *stream) {
    return guarded([&] {
        if (!gh || (k != 3 && k != 4)) throw Error{TG_ERR_INVALID_ARG, "k"};
        Graph &G = gh->g;
        cudaStream_t s = (cudaStream_t)stream;
        G.stream = s;
        tg::prepare_counting(G, k, s);
        tg::prepare_edges(G, k, s);
        const size_t pe_bytes = (size_t)G.m * tg::per_edge_slots(G.L, k) * sizeof(uint32_t);
        const size_t gl_bytes = (size_t)G.ngraphs * tg::global_slots(G.L, k) * sizeof(int64_t);
        bool pe_staged = false, gl_staged = false;
        uint32_t *pe = device_out(per_edge_out, pe_bytes, G.stage_pe, pe_staged);
        int64_t *gl = device_out(global_out, gl_bytes, G.stage_gl, gl_staged);
        TG_CK(cudaMemsetAsync(G.gacc.p, 0, (size_t)G.ngraphs * tg::global_slots(G.L, 4) * sizeof(unsigned long long), s));
        int64_t launches = tg::run_count(G, k, 0, G.m, pe, G.gacc.as<unsigned long long>(), true, s);
        if (gl) launches += tg::launch_finalize(G, k, gl, s);
        if (pe_staged && pe_bytes) TG_CK(cudaMemcpyAsync(per_edge_out, pe, pe_bytes, cudaMemcpyDeviceToHost, s));
        if (gl_staged) TG_CK(cudaMemcpyAsync(global_out, gl, gl_bytes, cudaMemcpyDeviceToHost, s));
        if (pe_staged || gl_staged) TG_CK(cudaStreamSynchronize(s));
        G.last_launches = launches;
    });
}

tg_status tg_count_handles(tg_graph *const *gs, int32_t ngraphs, int32_t k, int64_t *global_out, void *stream) {
    return guarded([&] {
        if (ngraphs < 0 || (ngraphs > 0 && (!gs || !global_out)) || (k != 3 && k != 4))
            throw Error{TG_ERR_INVALID_ARG, "args"};
        for (int32_t h = 0; h < ngraphs; ++h)
            if (!gs[h]) throw Error{TG_ERR_INVALID_ARG, "NULL handle"};
        int64_t off = 0;
        for (int32_t h = 0; h < ngraphs; ++h) {
            const Graph &G = gs[h]->g;
            const tg_status st = tg_count(gs[h], k, nullptr, global_out + off, stream);
            if (st != TG_OK) throw Error{st, "tg_count"};
            off += (int64_t)G.ngraphs * tg::global_slots(G.L, k);
        }
    });
}

tg_status tg_count_position_aware(tg_graph *gh, uint32_t *per_edge_out, int64_t *global_out, void *stream) {
    return guarded([&] {
        if (!gh) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        Graph &G = gh->g;
        cudaStream_t s = (cudaStream_t)stream;
        G.stream = s;
        tg::prepare_counting(G, 4, s);
        tg::prepare_edges(G, 4, s);
        tg::prepare_position_aware(G, s);
        const size_t pe_bytes = (size_t)G.m * G.pa.S * sizeof(uint32_t);
        const size_t gl_bytes = (size_t)G.ngraphs * G.pa.G * sizeof(int64_t);
        bool pe_staged = false, gl_staged = false;
        uint32_t *pe = device_out(per_edge_out, pe_bytes, G.stage_pe, pe_staged);
        int64_t *gl = device_out(global_out, gl_bytes, G.stage_gl, gl_staged);
        TG_CK(cudaMemsetAsync(G.pa_gacc.p, 0, (size_t)G.ngraphs * G.pa.G * sizeof(unsigned long long), s));
        struct Active {                                  // the epilogue writes position-aware rows meanwhile
            Graph &G;
            explicit Active(Graph &g) : G(g) { G.pa_active = true; }
            ~Active() { G.pa_active = false; }
        } active(G);
        int64_t launches = tg::run_count(G, 4, 0, G.m, pe, G.pa_gacc.as<unsigned long long>(), true, s);
        if (gl) launches += tg::launch_finalize_pa(G, gl, s);
        if (pe_staged && pe_bytes) TG_CK(cudaMemcpyAsync(per_edge_out, pe, pe_bytes, cudaMemcpyDeviceToHost, s));
        if (gl_staged) TG_CK(cudaMemcpyAsync(global_out, gl, gl_bytes, cudaMemcpyDeviceToHost, s));
        if (pe_staged || gl_staged) TG_CK(cudaStreamSynchronize(s));
        G.last_launches = launches;
    });
}

tg_status tg_count_range(tg_graph *gh, int32_t k, int64_t e_begin, int64_t e_end, uint32_t *per_edge_out,
                         int64_t *global_accum, void *stream) {
    return guarded([&] {
        if (!gh || (k != 3 && k != 4)) throw Error{TG_ERR_INVALID_ARG, "k"};
        Graph &G = gh->g;
        if (e_begin < 0 || e_end < e_begin || e_end > G.m) throw Error{TG_ERR_INVALID_ARG, "range"};
        cudaStream_t s = (cudaStream_t)stream;
        G.stream = s;
        tg::prepare_counting(G, k, s);
        tg::prepare_edges(G, k, s);
        int64_t launches = 0;
        const size_t pe_bytes = (size_t)(e_end - e_begin) * tg::per_edge_slots(G.L, k) * sizeof(uint32_t);
        const size_t gl_bytes = (size_t)G.ngraphs * tg::global_slots(G.L, k) * sizeof(int64_t);
        bool pe_staged = false, gl_staged = false;
        uint32_t *pe = device_out(per_edge_out, pe_bytes, G.stage_pe, pe_staged);
        int64_t *gl = device_out(global_accum, gl_bytes, G.stage_gl, gl_staged);
        if (gl_staged) TG_CK(cudaMemcpyAsync(gl, global_accum, gl_bytes, cudaMemcpyHostToDevice, s));
        unsigned long long *acc = gl ? reinterpret_cast<unsigned long long *>(gl) : nullptr;
        tg::DBuf scratch;
        scratch.owner = &G.stream;
        if (!acc) {
            scratch.alloc(gl_bytes);
            TG_CK(cudaMemsetAsync(scratch.p, 0, gl_bytes, s));
            acc = scratch.as<unsigned long long>();
        }
        launches += tg::run_count(G, k, e_begin, e_end, pe, acc, false, s);
        if (pe_staged && pe_bytes) TG_CK(cudaMemcpyAsync(per_edge_out, pe, pe_bytes, cudaMemcpyDeviceToHost, s));
        if (gl_staged) TG_CK(cudaMemcpyAsync(global_accum, gl, gl_bytes, cudaMemcpyDeviceToHost, s));
        if (pe_staged || gl_staged || scratch.p) TG_CK(cudaStreamSynchronize(s));
        G.last_launches = launches;
    });
}

tg_status tg_count_sparse(tg_graph *gh, int32_t k, int64_t *row_off, uint16_t *slot, uint32_t *value, int64_t cap,
                          int64_t *nnz, int64_t *global_out, void *stream) {
    return guarded([&] {
        if (!gh || (k != 3 && k != 4) || !nnz || cap < 0 || (!slot) != (!value))
            throw Error{TG_ERR_INVALID_ARG, "args"};
        for (const void *p : {(const void *)row_off, (const void *)slot, (const void *)value})
            if (p && !tg::is_device_pointer(p)) throw Error{TG_ERR_INVALID_ARG, "sparse arrays must be device memory"};
        Graph &G = gh->g;
        cudaStream_t s = (cudaStream_t)stream;
        G.stream = s;
        tg::prepare_counting(G, k, s);
        tg::prepare_edges(G, k, s);
        const size_t gl_bytes = (size_t)G.ngraphs * tg::global_slots(G.L, k) * sizeof(int64_t);
        bool gl_staged = false;
        int64_t *gl = device_out(global_out, gl_bytes, G.stage_gl, gl_staged);
        TG_CK(cudaMemsetAsync(G.gacc.p, 0, (size_t)G.ngraphs * tg::global_slots(G.L, 4) * sizeof(unsigned long long), s));
        bool fits = true;
        *nnz = tg::count_sparse(G, k, row_off, slot, value, cap, fits, s);
        if (gl) tg::launch_finalize(G, k, gl, s);
        if (gl_staged) TG_CK(cudaMemcpyAsync(global_out, gl, gl_bytes, cudaMemcpyDeviceToHost, s));
        TG_CK(cudaStreamSynchronize(s));
        if (slot && !fits) throw Error{TG_ERR_TOO_LARGE, "sparse capacity"};
    });
}

tg_status tg_graphlet_weights(tg_graph *gh, int32_t k, const uint32_t *per_edge_rows, int32_t block, int64_t rank,
                              int64_t *weights, int64_t *degree, void *stream) {
    return guarded([&] {
        if (!gh || (k != 3 && k != 4) || !per_edge_rows || !weights) throw Error{TG_ERR_INVALID_ARG, "args"};
        for (const void *p : {(const void *)per_edge_rows, (const void *)weights, (const void *)degree})
            if (p && !tg::is_device_pointer(p)) throw Error{TG_ERR_INVALID_ARG, "arrays must be device memory"};
        Graph &G = gh->g;
        G.stream = (cudaStream_t)stream;
        tg::launch_weights(G, k, per_edge_rows, block, rank, weights, degree, G.stream);
    });
}

tg_status tg_finalize_global(int32_t L, int32_t k, int32_t ngraphs, const int64_t *raw, int64_t *out) {
    return guarded([&] {
        check_types(L);
        if ((k != 3 && k != 4) || ngraphs < 0 || !raw || !out) throw Error{TG_ERR_INVALID_ARG, "args"};
        tg_layout_t lay;
        if (tg_layout(L, k, &lay) != TG_OK) throw Error{TG_ERR_INVALID_ARG, "layout"};
        bool bad = false;
        for (int32_t g = 0; g < ngraphs; ++g)
            for (int b = 0; b < 9; ++b)
                for (int64_t x = 0; x < lay.global_block_size[b]; ++x) {
                    const int64_t idx = g * lay.global_slots + lay.global_block_offset[b] + x;
                    if (raw[idx] % lay.graphlet_edges[b]) bad = true;
                    out[idx] = raw[idx] / lay.graphlet_edges[b];
                }
        if (bad) throw Error{TG_ERR_INTERNAL, "remainder"};
    });
}

tg_status tg_count_batch(tg_graph *gh, int32_t k, uint32_t *per_edge_out, int64_t *global_out, void *stream) {
    return guarded([&] {
        if (!gh || (k != 3 && k != 4) || !stream) throw Error{TG_ERR_INVALID_ARG, "k or stream"};
        if ((per_edge_out && !tg::is_device_pointer(per_edge_out)) || (global_out && !tg::is_device_pointer(global_out)))
            throw Error{TG_ERR_INVALID_ARG, "batched outputs must be device memory"};
        Graph &G = gh->g;
        cudaStream_t s = (cudaStream_t)stream;
        G.stream = s;
        const bool same = G.batch_exec && G.batch_k == k && G.batch_pe == per_edge_out && G.batch_gl == global_out &&
                          G.batch_stream == s;
        if (!same) {
            if (G.batch_exec) {
                cudaGraphExecDestroy(G.batch_exec);
                G.batch_exec = nullptr;
            }
            tg::prepare_counting(G, k, s);
            tg::prepare_edges(G, k, s);
            tg::prepare_capture(G, k, s);
            TG_CK(cudaStreamSynchronize(s));
            cudaGraph_t graph = nullptr;
            TG_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            int64_t launches = 0;
            try {
                TG_CK(cudaMemsetAsync(G.gacc.p, 0, (size_t)G.ngraphs * tg::global_slots(G.L, 4) * sizeof(unsigned long long), s));
                launches += tg::run_count(G, k, 0, G.m, per_edge_out, G.gacc.as<unsigned long long>(), true, s);
                if (global_out) launches += tg::launch_finalize(G, k, global_out, s);
            } catch (...) {
                cudaStreamEndCapture(s, &graph);
                if (graph) cudaGraphDestroy(graph);
                throw;
            }
            TG_CK(cudaStreamEndCapture(s, &graph));
            cudaError_t ie = cudaGraphInstantiate(&G.batch_exec, graph, 0);
            cudaGraphDestroy(graph);
            TG_CK(ie);
            G.batch_k = k;
            G.batch_pe = per_edge_out;
            G.batch_gl = global_out;
            G.batch_stream = s;
            G.last_launches = launches;
        }
        TG_CK(cudaGraphLaunch(G.batch_exec, s));
    });
}

tg_status tg_set_timing(tg_graph *gh, int32_t on) {
    return guarded([&] {
        if (!gh) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        gh->g.timing = on != 0;
    });
}

tg_status tg_set_work_counting(tg_graph *gh, int32_t on) {
    return guarded([&] {
        if (!gh) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        Graph &G = gh->g;
        if (on && !G.work.p) {
            G.work.alloc(sizeof(unsigned long long) * tg::kWorkSlots);
            TG_CK(cudaMemsetAsync(G.work.p, 0, sizeof(unsigned long long) * tg::kWorkSlots, G.stream));
        }
        G.work_on = on != 0;
    });
}

tg_status tg_get_work(tg_graph *gh, int64_t *out, int32_t n) {
    return guarded([&] {
        if (!gh || !out || n < 0) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        Graph &G = gh->g;
        unsigned long long h[tg::kWorkSlots] = {0};
        if (G.work.p) {
            TG_CK(cudaMemcpyAsync(h, G.work.p, sizeof(h), cudaMemcpyDeviceToHost, G.stream));
            TG_CK(cudaStreamSynchronize(G.stream));
            TG_CK(cudaMemsetAsync(G.work.p, 0, sizeof(h), G.stream));
        }
        for (int32_t k = 0; k < n; ++k) out[k] = k < tg::kWorkSlots ? (int64_t)h[k] : 0;
    });
}

tg_status tg_get_timing(tg_graph *gh, int32_t max, const char **names, double *ms, int64_t *launches, int32_t *n) {
    return guarded([&] {
        if (!gh || !n || max < 0) throw Error{TG_ERR_INVALID_ARG, "NULL"};
        Graph &G = gh->g;
        TG_CK(cudaStreamSynchronize(G.stream));
        for (auto &r : G.timer_pending) {
            float t = 0.f;
            TG_CK(cudaEventElapsedTime(&t, r.a, r.b));
            bool found = false;
            for (auto &tot : G.timer_totals)
                if (std::strcmp(tot.first, r.name) == 0) { tot.second.first += t; tot.second.second += 1; found = true; }
            if (!found) G.timer_totals.push_back({r.name, {(double)t, 1}});
            G.event_pool.push_back(r.a);
            G.event_pool.push_back(r.b);
        }
        G.timer_pending.clear();
        int32_t c = 0;
        for (auto &tot : G.timer_totals) {
            if (c < max) {
                if (names) names[c] = tot.first;
                if (ms) ms[c] = tot.second.first;
                if (launches) launches[c] = tot.second.second;
            }
            ++c;
        }
        *n = c < max ? c : max;
        G.timer_totals.clear();
    });
}

tg_status tg_query_status(tg_graph *gh) {
    if (!gh) return TG_ERR_INVALID_ARG;
    uint32_t v = 0;
    tg_status st = guarded([&] {
        Graph &G = gh->g;
        TG_CK(cudaStreamSynchronize(G.stream));
        TG_CK(cudaMemcpy(&v, G.status.p, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        TG_CK(cudaMemset(G.status.p, 0, sizeof(uint32_t)));
    });
    if (st != TG_OK) return st;
    if (v & tg::ST_INVALID_GRAPH) return TG_ERR_INVALID_GRAPH;
    if (v & tg::ST_TOO_LARGE) return TG_ERR_TOO_LARGE;
    if (v & tg::ST_TIMEOUT) return TG_ERR_TIMEOUT;
    if (v & tg::ST_INTERNAL) return TG_ERR_INTERNAL;
    if (v & tg::ST_OVERFLOW) return TG_ERR_OVERFLOW;
    return TG_OK;
}

const char *tg_last_error(void) { return tg::tl_last_error; }

const char *tg_status_string(tg_status s) {
    switch (s) {
        case TG_OK: return "ok";
        case TG_ERR_INVALID_ARG: return "invalid argument";
        case TG_ERR_INVALID_GRAPH: return "invalid graph (not a simple symmetric CSR, or a type >= L)";
        case TG_ERR_TOO_MANY_TYPES: return "number of types outside [1, TG_MAX_TYPES]";
        case TG_ERR_OOM: return "device memory exhausted";
        case TG_ERR_OVERFLOW: return "a per-edge count exceeded 2^32-1 and was saturated";
        case TG_ERR_TIMEOUT: return "a bounded device wait ran out";
        case TG_ERR_CUDA: return "CUDA runtime error";
        case TG_ERR_INTERNAL: return "internal consistency check failed";
        case TG_ERR_TOO_LARGE: return "graph exceeds an index-width limit";
    }
    return "unknown status";
}

}  // extern "C"
