// tg_static.cu -- tg_count3_static: typed 3-node counts that allocate nothing.
//
// Some callers cannot call cudaMalloc: services that hand all device memory
// to their own pool up front and forbid other allocations, code that runs
// while a CUDA graph is being captured (plain cudaMalloc/cudaFree cannot be
// captured), and latency-critical loops where cudaFree's implicit device
// synchronisation is not acceptable.  tg_count3_static serves them: the
// caller passes the graph and the output buffers, and the only working
// memory is the file-scope device array below, which every GPU that loads
// this library holds until the process exits.
//
// It computes the same per-edge typed 3-node counts and global typed 2- and
// 3-node totals as tg_count(k = 3) (typed triangles and 3-paths, Cor. 1-3),
// directly from the caller's CSR, without a tg_graph handle.
#include <algorithm>
#include <mutex>

#include "tg_host.hpp"

namespace tg {
namespace {

// ---- the static scratch --------------------------------------------------
// Limit: at most kStaticMaxNodes nodes per call.  Layout (int64 words):
//   [0, kStaticMaxNodes + 1)   per-row first edge id (exclusive prefix)
//   then kStaticGlobal words   raw global sums (unsigned)
//   then 1 word                status bits
constexpr int64_t kStaticMaxNodes = 1 << 20;
constexpr int kStaticGlobal = 36 + 2 * 120;     // G(8, k=3) = C(9,2) + 2 C(10,3)
constexpr int64_t kStaticWords = kStaticMaxNodes + 1 + kStaticGlobal + 1;
static __device__ __align__(256) unsigned long long g_static_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (set-up on first use).
unsigned long long *scratch_on_current_device() {
    int dev = 0;
    TG_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw Error{TG_ERR_INVALID_ARG, "device index"};
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        TG_CK(cudaGetSymbolAddress(&p, g_static_scratch));
        g_scratch_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    return g_scratch_ptr[dev];
}

__device__ __forceinline__ int mchoose(int n, int r) {      // C(n + r - 1, r)
    int v = 1;
    for (int k = 1; k <= r; ++k) v = v * (n + k - 1) / k;
    return v;
}
__device__ int rank_sorted(int L, int K, const int *s) {
    int r = 0, prev = 0;
    for (int k = 0; k < K; ++k) {
        for (int v = prev; v < s[k]; ++v) r += mchoose(L - v, K - k - 1);
        prev = s[k];
    }
    return r;
}

// Zero the global sums and the status word (the scratch keeps the previous
// call's contents otherwise).
__global__ void k_static_clear(unsigned long long *acc, int words) {
    for (int k = threadIdx.x; k < words; k += blockDim.x) acc[k] = 0;
}

// Row checks (sorted, in range, no self-loop) and the number of upper
// neighbours (v > u) of every row, written to first[u + 1].
__global__ void k_static_upper(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                               const int32_t *__restrict__ col, const uint8_t *__restrict__ ty, int L,
                               unsigned long long *first, unsigned long long *status) {
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u >= n) return;
    bool bad = ty[u] >= L || rp[u] < 0 || rp[u + 1] < rp[u] || rp[u + 1] > nnz;
    if ((u == 0 && rp[0] != 0) || (u == n - 1 && rp[n] != nnz)) bad = true;
    int64_t up = 0;
    for (int64_t k = rp[u]; k < rp[u + 1] && !bad; ++k) {
        const int32_t v = col[k];
        if (v < 0 || v >= n || v == u || (k > rp[u] && col[k - 1] >= v)) bad = true;
        up += v > u ? 1 : 0;
    }
    if (bad) atomicOr(status, (unsigned long long)ST_INVALID_GRAPH);
    first[u + 1] = (unsigned long long)up;
    if (u == 0) first[0] = 0;
}

// Symmetry: every entry v of row u needs the entry u in row v (one thread
// per entry, binary search in row v).  Runs after k_static_upper, so a
// graph it already rejected is skipped; indices stay clamped to [0, nnz).
__global__ void k_static_sym(int64_t n, int64_t nnz, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             unsigned long long *status) {
    if (*(volatile unsigned long long *)status != 0) return;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;                              // row u of entry k: rp[u] <= k < rp[u + 1]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (rp[mid] <= k) lo = mid; else hi = mid;
        }
        const int64_t u = lo;
        const int32_t v = col[k];
        if (v < 0 || v >= n) continue;                       // flagged by k_static_upper
        const int64_t end = rp[v + 1] < nnz ? rp[v + 1] : nnz;
        int64_t a = rp[v] > 0 ? rp[v] : 0, b = end;
        while (a < b) {
            const int64_t mid = (a + b) >> 1;
            if (col[mid] < u) a = mid + 1; else b = mid;
        }
        if (a >= end || col[a] != u) atomicOr(status, (unsigned long long)ST_INVALID_GRAPH);
    }
}

// Inclusive scan of first[1..n] in place (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_static_scan(int64_t n, unsigned long long *first) {
    __shared__ unsigned long long part[1024];
    unsigned long long carry = 0;
    for (int64_t base = 1; base <= n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        unsigned long long v = i <= n ? first[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            unsigned long long x = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += x;
            __syncthreads();
        }
        if (i <= n) first[i] = carry + part[threadIdx.x];
        const unsigned long long tot = part[1023];
        __syncthreads();
        carry += tot;
    }
}

// per-type counts of 32 entries of a row at once: lane t < L adds how many
// of the warp's valid entries have type t
__device__ __forceinline__ void count_types(bool valid, int type, int L, int lane, int &acc) {
    for (int t = 0; t < L; ++t) {
        const unsigned b = __ballot_sync(0xffffffffu, valid && type == t);
        if (lane == t) acc += __popc(b);
    }
}

// Warp per upper edge e = (u, v), u < v, in edge-id order: the row u with
// first[u] <= e < first[u + 1] by binary search; the typed degrees of u and
// v and the typed common neighbours (every entry of the shorter row searched
// in the longer one), all with ballots, so a hub row's edges spread over
// many warps.
__global__ void __launch_bounds__(256) k_static_tri3(int64_t n, int64_t m, const int64_t *__restrict__ rp,
                                                    const int32_t *__restrict__ col, const uint8_t *__restrict__ ty,
                                                    int L, const unsigned long long *__restrict__ first,
                                                    uint32_t *per_edge_out, unsigned long long *acc,
                                                    unsigned long long *status) {
    __shared__ unsigned long long hist[kStaticGlobal];
    __shared__ int s_bad;
    if (threadIdx.x == 0) {
        s_bad = *(volatile unsigned long long *)status != 0;
        if (!s_bad && first[n] != (unsigned long long)m) {   // upper entries must number the edges
            atomicOr(status, (unsigned long long)ST_INVALID_GRAPH);
            s_bad = 1;
        }
    }
    __syncthreads();
    if (s_bad) return;                                       // invalid rows: touch nothing (CTA-uniform)
    const int G = mchoose(L, 2) + 2 * mchoose(L, 3);
    for (int s = threadIdx.x; s < G; s += blockDim.x) hist[s] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; e < m; e += nw) {
        int64_t lo = 0, hi = n;                              // first[lo] <= e < first[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (first[mid] <= (unsigned long long)e) lo = mid; else hi = mid;
        }
        const int64_t u = lo;
        const int64_t ub = rp[u], ue = rp[u + 1];
        const int64_t start = ue - (int64_t)(first[u + 1] - first[u]);    // upper neighbours: a suffix
        const int32_t v = col[start + (e - (int64_t)first[u])];
        const int64_t vb = rp[v], ve = rp[v + 1];
        int du = 0, dv = 0, c = 0;                           // lane t < L: type-t counts
        for (int64_t k0 = ub; k0 < ue; k0 += 32) {
            const bool ok = k0 + lane < ue;
            count_types(ok, ok ? ty[col[k0 + lane]] : 0, L, lane, du);
        }
        for (int64_t k0 = vb; k0 < ve; k0 += 32) {
            const bool ok = k0 + lane < ve;
            count_types(ok, ok ? ty[col[k0 + lane]] : 0, L, lane, dv);
        }
        int64_t sb = ub, se = ue, lb = vb, le = ve;          // search the shorter row in the longer
        if (se - sb > le - lb) {
            int64_t x = sb; sb = lb; lb = x;
            x = se; se = le; le = x;
        }
        for (int64_t k0 = sb; k0 < se; k0 += 32) {
            bool hit = false;
            int32_t x = 0;
            if (k0 + lane < se) {
                x = col[k0 + lane];
                int64_t a = lb, b = le;
                while (a < b) {
                    const int64_t mid = (a + b) >> 1;
                    if (col[mid] < x) a = mid + 1; else b = mid;
                }
                hit = a < le && col[a] == x;
            }
            count_types(hit, hit ? ty[x] : 0, L, lane, c);
        }
        const int p = ty[u], q = ty[v];
        if (lane < L) {
            const int t = lane;
            const int64_t at = (int64_t)du - c - (q == t ? 1 : 0);      // |S_u^t|, S_u excludes v
            const int64_t bt = (int64_t)dv - c - (p == t ? 1 : 0);      // |S_v^t|
            if (at < 0 || bt < 0) {
                atomicOr(status, (unsigned long long)ST_INVALID_GRAPH);
            } else {
                if (per_edge_out) {
                    per_edge_out[e * 2 * L + t] = (uint32_t)(at + bt);
                    per_edge_out[e * 2 * L + L + t] = (uint32_t)c;
                }
                int ms[3] = {p, q, t};
                for (int x0 = 0; x0 < 2; ++x0)
                    for (int x1 = 0; x1 < 2 - x0; ++x1)
                        if (ms[x1] > ms[x1 + 1]) { int z = ms[x1]; ms[x1] = ms[x1 + 1]; ms[x1 + 1] = z; }
                const int r = rank_sorted(L, 3, ms);
                if (at + bt) atomicAdd(&hist[mchoose(L, 2) + r], (unsigned long long)(at + bt));
                if (c) atomicAdd(&hist[mchoose(L, 2) + mchoose(L, 3) + r], (unsigned long long)c);
            }
        }
        if (lane == 0) {
            int m2[2] = {p < q ? p : q, p < q ? q : p};
            atomicAdd(&hist[rank_sorted(L, 2, m2)], 1ull);
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < G; s += blockDim.x)
        if (hist[s]) atomicAdd(&acc[s], hist[s]);
}

// Global totals: edges / 1, 3-paths / 2, triangles / 3 (Sec. 6).
__global__ void k_static_finalize(int L, const unsigned long long *__restrict__ acc, int64_t *global_out,
                                  unsigned long long *status) {
    const int G = mchoose(L, 2) + 2 * mchoose(L, 3);
    for (int s = threadIdx.x; s < G; s += blockDim.x) {
        const int div = s < mchoose(L, 2) ? 1 : (s < mchoose(L, 2) + mchoose(L, 3) ? 2 : 3);
        if (acc[s] % div) atomicOr(status, (unsigned long long)ST_INTERNAL);
        global_out[s] = (int64_t)(acc[s] / div);
    }
}

__global__ void k_static_status(const unsigned long long *st, uint32_t *out) {
    if (threadIdx.x == 0) *out |= (uint32_t)*st;
}

}  // namespace
}  // namespace tg

extern "C" tg_status tg_count3_static(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                                      const uint8_t *node_types, int32_t L, uint32_t *per_edge_out,
                                      int64_t *global_out, uint32_t *device_status, void *stream) {
    try {
        using namespace tg;
        if (L < 1 || L > TG_MAX_TYPES) return TG_ERR_TOO_MANY_TYPES;
        if (n < 0 || nnz < 0 || (nnz & 1) || !row_ptr || (nnz > 0 && !col) || (n > 0 && !node_types))
            return TG_ERR_INVALID_ARG;
        if (n > kStaticMaxNodes || nnz >= ((int64_t)1 << 31)) return TG_ERR_TOO_LARGE;
        const void *ptrs[] = {row_ptr, col, node_types, per_edge_out, global_out, device_status};
        for (const void *p : ptrs)
            if (p && !is_device_pointer(p)) return TG_ERR_INVALID_ARG;   // device memory only: nothing to stage
        cudaStream_t s = (cudaStream_t)stream;
        unsigned long long *scratch = scratch_on_current_device();
        unsigned long long *first = scratch;
        unsigned long long *acc = scratch + kStaticMaxNodes + 1;
        unsigned long long *st = acc + kStaticGlobal;
        k_static_clear<<<1, 256, 0, s>>>(acc, kStaticGlobal + 1);
        if (n > 0) {
            k_static_upper<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, nnz, row_ptr, col, node_types, L, first, st);
            if (nnz > 0)
                k_static_sym<<<(unsigned)std::min<int64_t>((nnz + 255) / 256, 152 * 32), 256, 0, s>>>(n, nnz, row_ptr,
                                                                                                    col, st);
            k_static_scan<<<1, 1024, 0, s>>>(n, first);
            if (nnz > 0)
                k_static_tri3<<<(unsigned)std::min<int64_t>((nnz / 2 + 7) / 8, 152 * 16), 256, 0, s>>>(
                    n, nnz / 2, row_ptr, col, node_types, L, first, per_edge_out, acc, st);
        }
        if (global_out) k_static_finalize<<<1, 256, 0, s>>>(L, acc, global_out, st);
        if (device_status) k_static_status<<<1, 32, 0, s>>>(st, device_status);
        TG_CK(cudaGetLastError());
        return TG_OK;
    } catch (const tg::Error &e) {
        return e.status;
    } catch (...) {
        return TG_ERR_INTERNAL;
    }
}
