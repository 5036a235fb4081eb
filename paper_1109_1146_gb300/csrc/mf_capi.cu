// C ABI (include/mf.h) and the non-discharge kernels of the P-ARD sweep:
//   init      Init of Sec. 2 plus the terminal reduction;
//   fuse      label and flow fusion of Algorithm 2 on inter-region arcs;
//   gap_find  global gap of Sec. 5.1 on the histogram of boundary labels;
//   post      gap application, region activity for the next sweep;
//   cut       residual closures giving S_min and S_max.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "mf_internal.cuh"

using namespace mf;

struct mf_grid {
    int ndim = 0, conn = 0, H = 0, N = 0;
    bool host_state = false;                          // MF_STATE_HOST: planes and inputs in host memory
    Geom g{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int *cs = nullptr, *ct = nullptr, *nl = nullptr;  // stored inputs
    DevState st{};
    unsigned char *smin = nullptr, *tset = nullptr;
    void *cut_scratch = nullptr;                      // 2D cut: bit masks and sets
    void *br_scratch = nullptr;                       // boundary relabel (allocated at first use)
    int *h_br = nullptr;                              // pinned words of the boundary relabel
    int *warmF = nullptr, *warmFt = nullptr, *warmE = nullptr;  // projected initial flows (warm start)
    bool warm_ready = false;
    int warm_rounds = 0;
    // region reduction (Sec. 8): class codes, reduced inputs, device words
    // [counts[4], konst, err] and their pinned mirror
    unsigned char *red_codes = nullptr;
    int *red_cs = nullptr, *red_ct = nullptr, *red_nl = nullptr;
    unsigned long long *red_dev = nullptr, *h_red = nullptr;
    bool reduced = false;                             // the current solve runs on the reduced inputs
    long long red_konst = 0;                          // its constant (cut edges between the merged sets)
    int begin_active = -1;                            // active regions after mf_begin's relabel, -1: unknown
    bool begin_pending = false;                       // that relabel's counts are still in flight to h_ctr
    int *h_warm = nullptr;                            // pinned: the projection's flag words, read after a wait
    bool warm_pending = false;
    // CUDA graph of the sweep loop (opts.graph_loop)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;                // private stream the loop body is captured on
    int *loopctl = nullptr;                           // device loop state, see loop_ctl_kernel
    int *h_loop = nullptr;                            // pinned mirror
    int graph_key[5] = {-1, -1, -1, -1, -1};          // options baked into the graph
    Counters64 *c64 = nullptr;
    int *h_ctr = nullptr;                             // pinned mirror of st.ctr
    bool flow_cached = false;                         // stats.flow_value is that of the current state
    struct FinishHost {                               // pinned: results of the cut extraction, read after a sync
        int passes[2];
        long long f0;
        unsigned long long ft;
        Counters64 c;
    } *h_fin = nullptr;
    int *h_ctr_dv = nullptr;                          // device views of h_ctr and h_fin (kernels write them)
    FinishHost *h_fin_dv = nullptr;
    long long boundary = 0;
    bool caps_set = false, begun = false, finished = false;
    int sweep = 0;
    mf_opts opts{};
    mf_stats stats{};
    cudaEvent_t ev[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    long long launches = 0;
    std::string err;
};

static thread_local std::string g_static_err;

// the address a kernel reads p through (device memory, managed memory or
// pinned host memory), or nullptr if it cannot (pageable host memory)
static const void *device_view(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // an unknown pointer: clear the (non-sticky) error
        return nullptr;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged && a.type != cudaMemoryTypeHost) return nullptr;
    if (!a.devicePointer) return nullptr;
    // the offset of p inside its allocation carries over to the device view
    return (const char *)a.devicePointer + ((const char *)p - (const char *)(a.hostPointer ? a.hostPointer : a.devicePointer));
}

void mf::set_static_error(const std::string &m) { g_static_err = m; }

static mf_status fail(mf_grid *g, mf_status s, const std::string &m) {
    if (g) g->err = m;
    else g_static_err = m;
    return s;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(g, e_ == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                \
    } while (0)

// ---------------------------------------------------------------------------
// device helpers
__device__ __forceinline__ bool in_grid(const Geom &g, int x, int y, int z) {
    return x >= 0 && x < g.X && y >= 0 && y < g.Y && z >= 0 && z < g.Z;
}
__device__ __forceinline__ int region_of(const Geom &g, int x, int y, int z) {
    return ((z >> g.sz) * g.RY + (y >> g.sy)) * g.RX + (x >> g.sx);
}

// Init (Sec. 2): every s-link saturated, f := 0 on the rest, d := 0.  The part
// min(cs, ct) of a vertex is sent s -> v -> t at once (counted in flow0):
// exc = cs - min, tcap = ct - min.  cap[d] gets the edge capacity of arc d.
// Init of vertex v; returns min(cs, ct), its share of flow0
template <int CONN>
__device__ __forceinline__ int init_vertex(const Geom &g, const DevState &st, const int *__restrict__ cs,
                                           const int *__restrict__ ct, const int *__restrict__ nl, size_t v) {
    const size_t n = (size_t)g.n;
    const int x = (int)(v % g.X), y = (int)((v / g.X) % g.Y), z = (int)(v / ((size_t)g.X * g.Y));
    const int a = cs[v], b = ct[v], m = min(a, b);
    st.exc[v] = a - m;
    st.tcap[v] = b - m;
    st.lab[v] = 0;
#pragma unroll
    for (int d = 0; d < arcs_of(CONN); ++d) {
        const int dx = arc_dx(CONN, d), dy = arc_dy(CONN, d), dz = arc_dz(CONN, d);
        int c = 0;
        if (in_grid(g, x + dx, y + dy, z + dz)) {
            const size_t w = ((size_t)(z + dz) * g.Y + (y + dy)) * g.X + (x + dx);
            c = (d & 1) ? nl[(size_t)(d >> 1) * n + w] : nl[(size_t)(d >> 1) * n + v];
        }
        st.cap[(size_t)d * n + v] = c;
    }
    if (a - m > 0) st.active[region_of(g, x, y, z)] = 1;
    return m;
}

template <int CONN>
__global__ void init_kernel(const Geom g, const DevState st, const int *__restrict__ cs,
                            const int *__restrict__ ct, const int *__restrict__ nl) {
    long long part = 0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < (size_t)g.n; v += (size_t)gridDim.x * blockDim.x)
        part += init_vertex<CONN>(g, st, cs, ct, nl, v);
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part) atomicAdd((unsigned long long *)st.flow0, (unsigned long long)part);
}

// Init of many grids (a batch whose grids start cold): one launch resets the
// per-grid state (a block per grid: region flags, flow, counters, the label
// histogram with every boundary vertex at label 0), one runs Init over
// (grid, 64K vertices) units
struct InitJob {
    Geom g;
    DevState st;
    Counters64 *c64;
    const int *cs, *ct, *nl;
    int conn;
    int boundary;
};
constexpr int kInitChunk = 65536;
__global__ void batch_begin_reset_kernel(const InitJob *__restrict__ jobs) {
    const InitJob &J = jobs[blockIdx.x];
    const DevState &st = J.st;
    for (int r = threadIdx.x; r < J.g.nreg; r += blockDim.x) {
        st.active[r] = 0;
        st.disc[r] = 0;
        st.left_active[r] = 0;
    }
    for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x) st.hist[b] = b == 0 ? J.boundary : 0;
    for (int w = threadIdx.x; w < kCtrWords; w += blockDim.x) st.ctr[w] = 0;
    if (threadIdx.x == 0) {
        *st.flow_t = 0;
        *st.flow0 = 0;
        *J.c64 = Counters64{};
    }
}
__global__ void batch_init_kernel(const InitJob *__restrict__ jobs, const int2 *__restrict__ units, int nunits) {
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int2 w = units[u];
        const InitJob &J = jobs[w.x];
        const size_t v0 = (size_t)w.y * kInitChunk, v1 = min((size_t)J.g.n, v0 + kInitChunk);
        long long part = 0;
        for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            switch (J.conn) {
                case 4: part += init_vertex<4>(J.g, J.st, J.cs, J.ct, J.nl, v); break;
                case 8: part += init_vertex<8>(J.g, J.st, J.cs, J.ct, J.nl, v); break;
                default: part += init_vertex<6>(J.g, J.st, J.cs, J.ct, J.nl, v); break;
            }
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0 && part) atomicAdd((unsigned long long *)J.st.flow0, (unsigned long long)part);
    }
}

// Input validation of the capacities of vertex v: bit 0 negative value,
// bit 1 nonzero link leaving the grid, bit 2 possible int32 overflow.
template <int CONN>
__device__ __forceinline__ int validate_vertex(const Geom &g, const int *cs, const int *ct, const int *nl, size_t v) {
    const size_t n = (size_t)g.n;
    const int x = (int)(v % g.X), y = (int)((v / g.X) % g.Y), z = (int)(v / ((size_t)g.X * g.Y));
    int f = 0;
    if (cs[v] < 0 || ct[v] < 0) f |= 1;
    long long sum = cs[v];
#pragma unroll
    for (int d = 0; d < arcs_of(CONN); ++d) {
        const int dx = arc_dx(CONN, d), dy = arc_dy(CONN, d), dz = arc_dz(CONN, d);
        const bool ing = in_grid(g, x + dx, y + dy, z + dz);
        int c;
        if (d & 1) {
            if (!ing) continue;
            c = nl[(size_t)(d >> 1) * n + ((size_t)(z + dz) * g.Y + (y + dy)) * g.X + (x + dx)];
        } else {
            c = nl[(size_t)(d >> 1) * n + v];
            if (!ing && c != 0) f |= 2;
        }
        if (c < 0) f |= 1;
        if (c > INT_MAX / 2) f |= 4;
        sum += c;
    }
    if (sum > INT_MAX) f |= 4;
    return f;
}

template <int CONN>
__global__ void validate_kernel(const Geom g, const int *cs, const int *ct, const int *nl, int *flags) {
    int f = 0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < (size_t)g.n; v += (size_t)gridDim.x * blockDim.x)
        f |= validate_vertex<CONN>(g, cs, ct, nl, v);
    if (f) atomicOr(flags, f);
}

// the validation of many grids in one launch: units (grid, 64K vertices)
struct ValJob {
    Geom g;
    const int *cs, *ct, *nl;
    int conn;
};
constexpr int kValChunk = 65536;
__global__ void validate_batch_kernel(const ValJob *__restrict__ jobs, const int2 *__restrict__ units, int nunits,
                                      int *flags) {
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        const int2 w = units[u];
        const ValJob &J = jobs[w.x];
        const size_t v0 = (size_t)w.y * kValChunk, v1 = min((size_t)J.g.n, v0 + kValChunk);
        int f = 0;
        for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            switch (J.conn) {
                case 4: f |= validate_vertex<4>(J.g, J.cs, J.ct, J.nl, v); break;
                case 8: f |= validate_vertex<8>(J.g, J.cs, J.ct, J.nl, v); break;
                case 6: f |= validate_vertex<6>(J.g, J.cs, J.ct, J.nl, v); break;
                default: f |= 8;  // not a connectivity of the batched path
            }
        }
        f = __reduce_or_sync(0xffffffffu, f);
        if ((threadIdx.x & 31) == 0 && f) atomicOr(&flags[w.x], f);
    }
}

// A region is "touched" in a sweep when it or one of its neighbour regions
// (across a stencil arc) was discharged: only those can see their boundary
// flow, excess or labels change.
template <int CONN>
__device__ __forceinline__ bool region_touched(const Geom &g, const DevState &st, int r) {
    if (st.disc[r]) return true;
    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    if constexpr (is_paper(CONN)) {  // displacements up to 4 < tile width: the eight surrounding regions
        for (int qy = ry - 1; qy <= ry + 1; ++qy)
            for (int qx = rx - 1; qx <= rx + 1; ++qx)
                if (qx >= 0 && qx < g.RX && qy >= 0 && qy < g.RY && st.disc[qy * g.RX + qx]) return true;
        return false;
    } else {
#pragma unroll
        for (int d = 0; d < arcs_of(CONN); ++d) {
            const int qx = rx + arc_dx(CONN, d), qy = ry + arc_dy(CONN, d), qz = rz + arc_dz(CONN, d);
            if (qx < 0 || qx >= g.RX || qy < 0 || qy >= g.RY || qz < 0 || qz >= g.RZ) continue;
            if (st.disc[(qz * g.RY + qy) * g.RX + qx]) return true;
        }
        return false;
    }
}

__device__ __forceinline__ int hist_bin(int l) { return l < kHistBins ? l : kHistBins; }

// Flow and label fusion of Algorithm 2, gather form: every boundary vertex u
// updates only its own arcs and excess.  For an inter-region arc (u,w):
//   alpha(a,b) = [d'(a) <= d'(b) + 1];
//   u's push on (u,w) is kept iff alpha(w,u), w's push on (w,u) iff alpha(u,w);
//   a refused push goes back to its sender (residual and excess restored).
// Also commits the new boundary labels and keeps the histogram of boundary
// labels (Sec. 5.3: the global gap needs labels of B only) up to date.
// Fusion of one boundary vertex u = (lx, ly, lz) of region r (see above).
// The boundary-label histogram change is returned as (old bin, new bin), -1
// where there is none, for the caller to aggregate over its warp.
template <int CONN>
__device__ __forceinline__ void fuse_cell(const Geom &g, const DevState &st, const int r, const int lx, const int ly,
                                          const int lz, const bool discr, int &bin_old, int &bin_new) {
    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    const size_t n = (size_t)g.n;
    const int x = rx * g.tx + lx, y = ry * g.ty + ly, z = rz * g.tz + lz;
    bin_old = bin_new = -1;
    if (!in_grid(g, x, y, z)) return;
    const size_t u = ((size_t)z * g.Y + y) * g.X + x;
    bool boundary = false;
    int back_total = 0;
    int du = -1;
#pragma unroll
    for (int d = 0; d < arcs_of(CONN); ++d) {
        const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d), wz = z + arc_dz(CONN, d);
        if (!in_grid(g, wx, wy, wz)) continue;
        const int rw = region_of(g, wx, wy, wz);
        if (rw == r) continue;
        if (!boundary) {
            boundary = true;
            du = discr ? st.lab_next[u] : st.lab[u];
        }
        const size_t w = ((size_t)wz * g.Y + wy) * g.X + wx;
        const bool discw = st.disc[rw];
        const int pu = discr ? st.bout[(size_t)d * n + u] : 0;
        const int pw = discw ? st.bout[(size_t)(d ^ 1) * n + w] : 0;
        if (!(pu | pw)) continue;  // no flow crossed this arc: nothing to accept or return
        const int dw = discw ? st.lab_next[w] : st.lab[w];
        const int back = (dw <= du + 1 ? 0 : pu) + (du <= dw + 1 ? pw : 0);
        if (back) {
            st.cap[(size_t)d * n + u] += back;
            back_total += back;
        }
    }
    if (!boundary) return;
    if (back_total) st.exc[u] += back_total;
    if (discr) {
        const int old = st.lab[u];
        if (old != du) {
            if (old < g.dinf) bin_old = hist_bin(old);
            if (du < g.dinf) bin_new = hist_bin(du);
            st.lab[u] = du;
        }
    }
}

// Histogram updates of a warp: lanes naming the same bin send one atomic
// with their count (a sweep moves many boundary labels between the same few
// bins, and per-vertex atomics on them serialise).
__device__ __forceinline__ void hist_update_warp(int *hist, int bin_old, int bin_new) {
    const int lane = threadIdx.x & 31;
    const unsigned mo = __match_any_sync(0xffffffffu, bin_old);
    if (bin_old >= 0 && lane == __ffs(mo) - 1) atomicSub(&hist[bin_old], __popc(mo));
    const unsigned mn = __match_any_sync(0xffffffffu, bin_new);
    if (bin_new >= 0 && lane == __ffs(mn) - 1) atomicAdd(&hist[bin_new], __popc(mn));
}

// The cells on the surface of a tile, enumerated directly: in 2D the top and
// bottom rows, then the left and right columns without their corners; in 3D
// the two z faces, then the two y faces without their z edge rows, then the
// two x faces without their y and z edges.  Tiles are at least 2 cells wide.
__device__ __forceinline__ int surface_cells(const Geom &g, bool is3d) {
    if (!is3d) return 2 * g.tx + 2 * (g.ty - 2);
    return 2 * g.tx * g.ty + 2 * g.tx * (g.tz - 2) + 2 * (g.ty - 2) * (g.tz - 2);
}
__device__ __forceinline__ void surface_cell(const Geom &g, bool is3d, int p, int &lx, int &ly, int &lz) {
    if (!is3d) {
        lz = 0;
        if (p < g.tx) { lx = p; ly = 0; }
        else if (p < 2 * g.tx) { lx = p - g.tx; ly = g.ty - 1; }
        else if (p < 2 * g.tx + g.ty - 2) { lx = 0; ly = 1 + p - 2 * g.tx; }
        else { lx = g.tx - 1; ly = 1 + p - 2 * g.tx - (g.ty - 2); }
        return;
    }
    const int A = g.tx * g.ty;
    if (p < 2 * A) {
        lz = p < A ? 0 : g.tz - 1;
        const int q = p < A ? p : p - A;
        lx = q % g.tx;
        ly = q / g.tx;
        return;
    }
    p -= 2 * A;
    const int Bf = g.tx * (g.tz - 2);
    if (p < 2 * Bf) {
        ly = p < Bf ? 0 : g.ty - 1;
        const int q = p < Bf ? p : p - Bf;
        lx = q % g.tx;
        lz = 1 + q / g.tx;
        return;
    }
    p -= 2 * Bf;
    const int Cf = (g.ty - 2) * (g.tz - 2);
    lx = p < Cf ? 0 : g.tx - 1;
    const int q = p < Cf ? p : p - Cf;
    ly = 1 + q % (g.ty - 2);
    lz = 1 + q / (g.ty - 2);
}

// region_touched for a whole warp in one round of loads: lane d reads the
// flag of the neighbour region across arc d (the 3 x 3 block of regions for
// the Sec. 7.1 stencils), the next lane the region's own
template <int CONN>
__device__ __forceinline__ bool region_touched_warp(const Geom &g, const DevState &st, int r) {
    const int lane = threadIdx.x & 31;
    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    bool f = false;
    if constexpr (is_paper(CONN)) {
        if (lane < 9) {
            const int qx = rx + lane % 3 - 1, qy = ry + lane / 3 - 1;
            if (qx >= 0 && qx < g.RX && qy >= 0 && qy < g.RY) f = st.disc[qy * g.RX + qx] != 0;
        }
    } else {
        if (lane < CONN) {
            const int qx = rx + arc_dx(CONN, lane), qy = ry + arc_dy(CONN, lane), qz = rz + arc_dz(CONN, lane);
            if (qx >= 0 && qx < g.RX && qy >= 0 && qy < g.RY && qz >= 0 && qz < g.RZ)
                f = st.disc[(qz * g.RY + qy) * g.RX + qx] != 0;
        } else if (lane == CONN) {
            f = st.disc[r] != 0;
        }
    }
    return __any_sync(0xffffffffu, f);
}

// Fusion of one touched region by one warp over the tile surface (only
// surface cells can be boundary vertices).
template <int CONN>
__device__ __forceinline__ void fuse_region_warp(const Geom &g, const DevState &st, const int r) {
    if (!region_touched_warp<CONN>(g, st, r)) return;
    const bool discr = st.disc[r];
    // boundary vertices lie on the tile surface, or (the longer displacements
    // of Sec. 7.1) anywhere in a band of the stencil's width: all cells then
    const int P = is_paper(CONN) ? g.tx * g.ty : surface_cells(g, CONN == 6);
    for (int p0 = 0; p0 < P; p0 += 32) {  // whole warp per step: the histogram update is a warp operation
        const int p = p0 + (threadIdx.x & 31);
        int bo = -1, bn = -1;
        if (p < P) {
            int lx, ly, lz;
            if (is_paper(CONN)) { lx = p & (g.tx - 1); ly = p >> g.sx; lz = 0; }
            else surface_cell(g, CONN == 6, p, lx, ly, lz);
            fuse_cell<CONN>(g, st, r, lx, ly, lz, discr, bo, bn);
        }
        hist_update_warp(st.hist, bo, bn);
    }
}

// Activity of one region after the fusion (one warp): with a gap, every label
// g < d < d_inf of the tile becomes d_inf first (all cells); a touched region
// is active if its discharge left interior excess (left_active) or a surface
// vertex has excess below d_inf.
template <int CONN>
__device__ __forceinline__ void post_region_warp(const Geom &g, const DevState &st, const int r, const int gap) {
    const int lane = threadIdx.x & 31;
    const bool touched = region_touched_warp<CONN>(g, st, r);
    if (!touched && gap == 0) return;
    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    int act = touched ? st.left_active[r] : 0;
    if (gap > 0) {
        const int V = g.tx * g.ty * g.tz;
        for (int i = lane; i < V; i += 32) {
            const int lx = i & (g.tx - 1), ly = (i >> g.sx) & (g.ty - 1), lz = i >> (g.sx + g.sy);
            const int x = rx * g.tx + lx, y = ry * g.ty + ly, z = rz * g.tz + lz;
            if (!in_grid(g, x, y, z)) continue;
            const size_t u = ((size_t)z * g.Y + y) * g.X + x;
            int l = st.lab[u];
            if (l > gap && l < g.dinf) {
                l = g.dinf;
                st.lab[u] = l;
            }
            constexpr int R = radius_of(CONN);
            const bool border = lx < R || lx >= g.tx - R || ly < R || ly >= g.ty - R ||
                                (CONN == 6 && (lz == 0 || lz == g.tz - 1));
            if (touched && border && l < g.dinf && st.exc[u] > 0) act = 1;
        }
    } else {
        const int P = is_paper(CONN) ? g.tx * g.ty : surface_cells(g, CONN == 6);
        for (int p = lane; p < P && !act; p += 32) {
            int lx, ly, lz;
            if (is_paper(CONN)) { lx = p & (g.tx - 1); ly = p >> g.sx; lz = 0; }
            else surface_cell(g, CONN == 6, p, lx, ly, lz);
            const int x = rx * g.tx + lx, y = ry * g.ty + ly, z = rz * g.tz + lz;
            if (!in_grid(g, x, y, z)) continue;
            const size_t u = ((size_t)z * g.Y + y) * g.X + x;
            if (st.exc[u] > 0 && st.lab[u] < g.dinf) act = 1;
        }
    }
    act = __any_sync(0xffffffffu, act);
    if (lane == 0 && touched) {
        st.active[r] = (unsigned char)act;
        if (act) atomicAdd(&st.ctr[kActiveRegions], 1);
    }
}

// single 3D grid: a warp per region, grid-stride
template <int CONN>
__global__ void fuse_warp_kernel(const Geom g, const DevState st) {
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < g.nreg; r += nw)
        fuse_region_warp<CONN>(g, st, r);
}
template <int CONN>
__global__ void post_warp_kernel(const Geom g, const DevState st) {
    const int gap = st.ctr[kGap];
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < g.nreg; r += nw)
        post_region_warp<CONN>(g, st, r, gap);
}

// Global gap (Sec. 5.1, with the boundary-label histogram of Sec. 5.3): the
// smallest g > 0 below the highest boundary label with no boundary vertex
// labelled g.  Every vertex with g < d < d_inf cannot reach t.  The bins
// above g are emptied (those labels become d_inf).
__device__ __forceinline__ void gap_find_body(const DevState &st) {
    __shared__ int s_hi, s_g;
    if (threadIdx.x == 0) { s_hi = 0; s_g = INT_MAX; }
    __syncthreads();
    int hi = 0;
    for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x)
        if (st.hist[b] > 0) hi = max(hi, b);
    atomicMax(&s_hi, hi);
    __syncthreads();
    const int top = s_hi;  // labels >= kHistBins share the last bin: never a gap there
    int gmin = INT_MAX;
    for (int b = 1 + threadIdx.x; b < top && b < kHistBins; b += blockDim.x)
        if (st.hist[b] == 0) gmin = min(gmin, b);
    atomicMin(&s_g, gmin);
    __syncthreads();
    const int gap = s_g == INT_MAX ? 0 : s_g;
    if (threadIdx.x == 0) st.ctr[kGap] = gap;
    if (gap > 0)
        for (int b = gap + 1 + threadIdx.x; b <= kHistBins; b += blockDim.x) st.hist[b] = 0;
}

__global__ void gap_find_kernel(const DevState st) { gap_find_body(st); }

// ---- 2D fusion and activity over perimeter items -----------------------------
// One thread per (region, perimeter slot): only tile perimeters hold boundary
// vertices, so the 2D sweep kernels walk 2 tx + 2 (ty - 2) slots per region
// instead of whole tiles (a warp covers one region's perimeter, and its lanes
// share the region-touched test through the cache).
__device__ __forceinline__ void perimeter_xy(int p, int tx, int ty, int &lx, int &ly) {
    if (p < tx) { lx = p; ly = 0; }
    else if (p < 2 * tx) { lx = p - tx; ly = ty - 1; }
    else if (p < 2 * tx + ty - 2) { lx = 0; ly = 1 + p - 2 * tx; }
    else { lx = tx - 1; ly = 1 + p - 2 * tx - (ty - 2); }
}

__device__ __forceinline__ int perimeter_slots(const Geom &g) { return 2 * g.tx + 2 * (g.ty - 2); }

// Algorithm 2's fusion for one boundary vertex u of region r (gather form;
// see fuse_region); also restarts the activity of a touched region from the
// excess its discharge left inside the tile.
template <int CONN>
__global__ void fuse2d_kernel(const Geom g, const DevState st) {
    const int P = perimeter_slots(g);
    const long long items = (long long)g.nreg * P;
    const int lane = threadIdx.x & 31;
    // warp-uniform steps (the histogram update is a warp operation)
    for (long long k0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x - lane); k0 < items;
         k0 += (long long)gridDim.x * blockDim.x) {
        const long long k = k0 + lane;
        int bo = -1, bn = -1;
        if (k < items) {
            const int r = (int)(k / P), p = (int)(k % P);
            if (region_touched<CONN>(g, st, r)) {
                if (p == 0) st.active[r] = st.left_active[r];
                int lx, ly;
                perimeter_xy(p, g.tx, g.ty, lx, ly);
                fuse_cell<CONN>(g, st, r, lx, ly, 0, st.disc[r] != 0, bo, bn);
            }
        }
        hist_update_warp(st.hist, bo, bn);
    }
}

// Activity after the fusion: a touched region is active if its discharge left
// interior excess or a perimeter vertex has excess below d_inf.  With a gap,
// first every label g < d < d_inf in the grid becomes d_inf (all vertices).
template <int CONN>
__global__ void post2d_kernel(const Geom g, const DevState st) {
    const int gap = st.ctr[kGap];
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (gap == 0) {
        const int P = perimeter_slots(g);
        const long long items = (long long)g.nreg * P;
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < items; k += stride) {
            const int r = (int)(k / P), p = (int)(k % P);
            int lx, ly;
            perimeter_xy(p, g.tx, g.ty, lx, ly);
            const int x = (r % g.RX) * g.tx + lx, y = (r / g.RX) * g.ty + ly;
            if (x >= g.X || y >= g.Y) continue;
            const size_t u = (size_t)y * g.X + x;
            if (st.exc[u] > 0 && st.lab[u] < g.dinf && region_touched<CONN>(g, st, r)) st.active[r] = 1;
        }
    } else {
        for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < (long long)g.n; v += stride) {
            const int x = (int)(v % g.X), y = (int)(v / g.X);
            int l = st.lab[v];
            if (l > gap && l < g.dinf) {
                l = g.dinf;
                st.lab[v] = l;
            }
            const int lx = x & (g.tx - 1), ly = y & (g.ty - 1);
            if (lx != 0 && lx != g.tx - 1 && ly != 0 && ly != g.ty - 1) continue;
            const int r = (y >> g.sy) * g.RX + (x >> g.sx);
            if (l < g.dinf && st.exc[v] > 0 && region_touched<CONN>(g, st, r)) st.active[r] = 1;
        }
    }
}

// count the active regions for the host, reset the per-sweep flags
__global__ void finish_flags_kernel(const DevState st, int nreg) {
    int c = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) {
        c += st.active[r] != 0;
        st.disc[r] = 0;
        st.left_active[r] = 0;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st.ctr[kActiveRegions], c);
}

// ---- device-side sweep loop (CUDA graph with a conditional while node) ------
// loopctl: [0] sweeps done (the next sweep's index), [1] sweeps that found a
// gap, [2] sweep cap, [3] relabel period P (0: none), [4] active regions
// after the last sweep, [5] error flag of the last sweep, [6] an extra sweep
// count F after which to stop (0: none).  The loop continues while no error
// was raised, some region is active, the cap is not reached and the sweep
// count is neither a multiple of P nor F (the host then runs the relabel due
// and relaunches the graph).
enum { kLoopSweep = 0, kLoopGaps, kLoopCap, kLoopPeriod, kLoopActive, kLoopError, kLoopFirst, kLoopWords = 8 };

__device__ __forceinline__ bool loop_stop_at(const int *lc, int s) {
    const int P = lc[kLoopPeriod], F = lc[kLoopFirst];
    return (P > 0 && s % P == 0) || (F > 0 && s == F);
}

__global__ void loop_ctl_kernel(const int *ctr, int *lc, cudaGraphConditionalHandle handle) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int active = ctr[kActiveRegions], err = ctr[kError], gap = ctr[kGap];
    const int s = lc[kLoopSweep] + 1;
    lc[kLoopSweep] = s;
    if (gap > 0) lc[kLoopGaps] += 1;
    lc[kLoopActive] = active;
    lc[kLoopError] = err;
    const bool cont = !err && active > 0 && s < lc[kLoopCap] && !loop_stop_at(lc, s);
    cudaGraphSetConditional(handle, cont ? 1u : 0u);
}

// the batch's loop control: any = some instance still has an active region
__global__ void batch_loop_ctl_kernel(const int *any, int *lc, cudaGraphConditionalHandle handle) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int s = lc[kLoopSweep] + 1;
    lc[kLoopSweep] = s;
    lc[kLoopActive] = *any;
    cudaGraphSetConditional(handle, (*any && s < lc[kLoopCap] && !loop_stop_at(lc, s)) ? 1u : 0u);
}

// ---- batched sweep kernels: one block per (instance, region) of the batch table
__global__ void batch_reset_kernel(const Inst *insts, const unsigned char *done, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        if (!done[i]) {
            int *c = insts[i].st.ctr;
            c[kActiveRegions] = 0;
            c[kGap] = 0;
        }
}

// work lists of the active regions, one list per kernel type
// (warp-uniform steps: the lanes that queue items of one kernel type take
// their slots with one atomic; neighbouring regions share an instance and so
// a type, and one atomic per item on the few counters serialised)
__global__ void batch_items_kernel(const Inst *insts, const int2 *regs, int nregs, const unsigned char *done,
                                   const int *type_of, int cap_per_type, int2 *items, int *cnt) {
    const int lane = threadIdx.x & 31;
    for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x - lane); i0 < nregs; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + lane;
        int t = -1;
        int2 w = make_int2(0, 0);
        if (i < nregs) {
            w = regs[i];
            if (!done[w.x] && insts[w.x].st.active[w.y]) t = type_of[w.x];
        }
        const unsigned m = __match_any_sync(0xffffffffu, t);
        const int leader = __ffs(m) - 1;
        int base = 0;
        if (t >= 0 && lane == leader) base = atomicAdd(&cnt[t], __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (t >= 0) items[(size_t)t * cap_per_type + base + __popc(m & ((1u << lane) - 1u))] = w;
    }
}

// batched fusion / activity: a warp per region of the whole batch, grid-stride
template <int CONN>
__global__ void fuse_batch_kernel(const Inst *insts, const int2 *regs, int nregs, const unsigned char *done) {
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nregs; i += nw) {
        const int2 w = regs[i];
        if (done[w.x] || insts[w.x].conn != CONN) continue;
        fuse_region_warp<CONN>(insts[w.x].g, insts[w.x].st, w.y);
    }
}

__global__ void gap_find_batch_kernel(const Inst *insts, const unsigned char *done) {
    if (done[blockIdx.x]) return;
    gap_find_body(insts[blockIdx.x].st);
}

template <int CONN>
__global__ void post_batch_kernel(const Inst *insts, const int2 *regs, int nregs, const unsigned char *done) {
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nregs; i += nw) {
        const int2 w = regs[i];
        if (done[w.x] || insts[w.x].conn != CONN) continue;
        post_region_warp<CONN>(insts[w.x].g, insts[w.x].st, w.y, insts[w.x].st.ctr[kGap]);
    }
}

__global__ void clear_batch_kernel(const Inst *insts, const int2 *regs, int nregs, const unsigned char *done) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nregs; i += gridDim.x * blockDim.x) {
        const int2 w = regs[i];
        if (done[w.x]) continue;
        insts[w.x].st.disc[w.y] = 0;
        insts[w.x].st.left_active[w.y] = 0;
    }
}

// per instance: finished when no region is active; an error also ends it
__global__ void batch_end_kernel(const Inst *insts, unsigned char *done, int *sweeps, int *any, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        if (done[i]) continue;
        const int *c = insts[i].st.ctr;
        sweeps[i] += 1;
        if (c[kActiveRegions] == 0 || c[kError]) done[i] = 1;
        else atomicAdd(any, 1);
    }
}

// after a relabel of the batch: instances left without an active region are
// done (as a single solve stops there); any = instances still active
__global__ void batch_relabel_end_kernel(const Inst *insts, unsigned char *done, int *any, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        if (done[i]) continue;
        if (insts[i].st.ctr[kActiveRegions] == 0) done[i] = 1;
        else atomicAdd(any, 1);
    }
}

// per-sweep flags are cleared after post has read them
__global__ void clear_flags_kernel(const DevState st, int nreg) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) {
        st.disc[r] = 0;
        st.left_active[r] = 0;
    }
}

// histogram at Init: every boundary vertex has label 0
__global__ void hist_init_kernel(const DevState st, int nb) {
    if (threadIdx.x == 0 && blockIdx.x == 0) st.hist[0] = nb;
}

__global__ void cut_seed_kernel(const Geom g, const DevState st, unsigned char *smin, unsigned char *tset) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < (size_t)g.n; v += (size_t)gridDim.x * blockDim.x) {
        smin[v] = st.exc[v] > 0;
        tset[v] = st.tcap[v] > 0;
    }
}

// One pass of a residual closure, region by region (pull form: a block only
// writes vertices of its own region).  fwd = 1: w joins if some member u has a
// residual arc u -> w (S_min, the closure of {e > 0}); fwd = 0: u joins if it
// has a residual arc u -> w into the set (vertices reaching t).
template <int CONN>
__global__ void cut_pass_kernel(const Geom g, const DevState st, unsigned char *set, int fwd) {
    extern __shared__ unsigned char s_in[];
    const int r = blockIdx.x;
    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    const int TX = g.tx, TY = g.ty, V = g.tx * g.ty * g.tz;
    const size_t n = (size_t)g.n;
    for (int i = threadIdx.x; i < V; i += blockDim.x) {
        const int x = rx * TX + i % TX, y = ry * TY + (i / TX) % TY, z = rz * g.tz + i / (TX * TY);
        s_in[i] = in_grid(g, x, y, z) ? set[((size_t)z * g.Y + y) * g.X + x] : 0;
    }
    __syncthreads();
    int grew = 0;
    for (bool first = true;; first = false) {
        int ch = 0;
        for (int i = threadIdx.x; i < V; i += blockDim.x) {
            if (s_in[i]) continue;
            const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
            const int x = rx * TX + lx, y = ry * TY + ly, z = rz * g.tz + lz;
            if (!in_grid(g, x, y, z)) continue;
            const size_t u = ((size_t)z * g.Y + y) * g.X + x;
#pragma unroll
            for (int d = 0; d < arcs_of(CONN); ++d) {
                const int dx = arc_dx(CONN, d), dy = arc_dy(CONN, d), dz = arc_dz(CONN, d);
                const int wx = x + dx, wy = y + dy, wz = z + dz;
                if (!in_grid(g, wx, wy, wz)) continue;
                const size_t w = ((size_t)wz * g.Y + wy) * g.X + wx;
                const int nlx = lx + dx, nly = ly + dy, nlz = lz + dz;
                const bool intile = nlx >= 0 && nlx < TX && nly >= 0 && nly < TY && nlz >= 0 && nlz < g.tz;
                if (!intile && !first) continue;  // other regions: read once per pass
                const unsigned char member = intile ? s_in[i + dx + dy * TX + dz * TX * TY] : set[w];
                if (!member) continue;
                const int res = fwd ? st.cap[(size_t)(d ^ 1) * n + w] : st.cap[(size_t)d * n + u];
                if (res > 0) {
                    s_in[i] = 1;
                    ch = 1;
                    break;
                }
            }
        }
        grew |= ch;
        if (!__syncthreads_or(ch)) break;
    }
    if (__syncthreads_or(grew)) {
        for (int i = threadIdx.x; i < V; i += blockDim.x) {
            const int x = rx * TX + i % TX, y = ry * TY + (i / TX) % TY, z = rz * g.tz + i / (TX * TY);
            if (!in_grid(g, x, y, z) || !s_in[i]) continue;
            const size_t u = ((size_t)z * g.Y + y) * g.X + x;
            if (!set[u]) set[u] = 1;
        }
        if (threadIdx.x == 0) st.ctr[kChanged] = 1;
    }
}

__global__ void complement_kernel(unsigned char *a, size_t n) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
        a[v] = !a[v];
}

// ---------------------------------------------------------------------------
// host side
static int grid_blocks(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    return (int)std::min<size_t>(std::max<size_t>(b, 1), device_sms() * 16);
}

template <int CONN>
static cudaError_t launch_init(mf_grid *h) {
    const int *cs = h->reduced ? h->red_cs : h->cs, *ct = h->reduced ? h->red_ct : h->ct;
    const int *nl = h->reduced ? h->red_nl : h->nl;
    init_kernel<CONN><<<grid_blocks(h->g.n, 256), 256, 0, h->stream>>>(h->g, h->st, cs, ct, nl);
    return cudaGetLastError();
}
template <int CONN>
static cudaError_t launch_validate(mf_grid *h, int *flags) {
    validate_kernel<CONN><<<grid_blocks(h->g.n, 256), 256, 0, h->stream>>>(h->g, h->cs, h->ct, h->nl, flags);
    return cudaGetLastError();
}
template <int CONN>
static cudaError_t launch_fuse_post(mf_grid *h, bool gap_on, cudaStream_t st) {
    if (CONN != 6 && !is_paper(CONN)) {
        const long long items = (long long)h->g.nreg * (2 * h->g.tx + 2 * (h->g.ty - 2));
        const int fb = (int)std::min<long long>((items + 255) / 256, device_sms() * 8);
        fuse2d_kernel<CONN><<<fb, 256, 0, st>>>(h->g, h->st);
        if (gap_on) gap_find_kernel<<<1, 1024, 0, st>>>(h->st);
        post2d_kernel<CONN><<<device_sms() * 8, 256, 0, st>>>(h->g, h->st);
        finish_flags_kernel<<<(h->g.nreg + 255) / 256, 256, 0, st>>>(h->st, h->g.nreg);
        return cudaGetLastError();
    }
    const int wb = (int)std::min<long long>(((long long)h->g.nreg + 7) / 8, (long long)device_sms() * 8);
    fuse_warp_kernel<CONN><<<wb, 256, 0, st>>>(h->g, h->st);
    if (gap_on) gap_find_kernel<<<1, 1024, 0, st>>>(h->st);
    post_warp_kernel<CONN><<<wb, 256, 0, st>>>(h->g, h->st);
    clear_flags_kernel<<<(h->g.nreg + 255) / 256, 256, 0, st>>>(h->st, h->g.nreg);
    return cudaGetLastError();
}
template <int CONN>
static cudaError_t launch_cut_pass(mf_grid *h, unsigned char *set, int fwd, cudaStream_t st) {
    const int V = h->g.tx * h->g.ty * h->g.tz;
    cut_pass_kernel<CONN><<<h->g.nreg, 256, V, st>>>(h->g, h->st, set, fwd);
    return cudaGetLastError();
}

#define DISPATCH(conn, fn, ...)                                                                              \
    ((conn) == 4 ? fn<4>(__VA_ARGS__) : (conn) == 8 ? fn<8>(__VA_ARGS__) : (conn) == 6 ? fn<6>(__VA_ARGS__)    \
     : (conn) == 108 ? fn<108>(__VA_ARGS__) : (conn) == 112 ? fn<112>(__VA_ARGS__)                            \
     : (conn) == 116 ? fn<116>(__VA_ARGS__) : (conn) == 120 ? fn<120>(__VA_ARGS__)                            \
     : (conn) == 124 ? fn<124>(__VA_ARGS__) : fn<128>(__VA_ARGS__))

// Optimality certificate of a finished solve, from the original capacities:
// counts violations of the capacity constraints (r(v,w) >= 0 and
// r(v,w) + r(w,v) = 2 c(v,w); no residual arc leaving the grid), of the sink
// residual (0 <= c_f(v,t) <= ct - min(cs,ct)) and of conservation
// (e(v) = cs' - f(v,t) - sum_w f(v,w) and e(v) >= 0), and sums the capacity
// of the cut (S, V \ S) for S = S_min: cs over V \ S, ct over S, c(v,w) over
// arcs from S to V \ S, and the flow into t, min(cs,ct) + ct' - c_f(v,t).
// Weak duality: a feasible preflow whose sink inflow equals the capacity of
// some cut is a maximum flow and the cut a minimum cut (Sec. 2).
template <int CONN>
__global__ void certify_kernel(const Geom g, const DevState st, const int *__restrict__ cs, const int *__restrict__ ct,
                               const int *__restrict__ nl, const unsigned char *__restrict__ S,
                               unsigned long long *sums) {
    const size_t n = (size_t)g.n;
    unsigned long long cut = 0, tin = 0, bad = 0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % g.X), y = (int)((v / g.X) % g.Y), z = (int)(v / ((size_t)g.X * g.Y));
        const int a = cs[v], b = ct[v], m = min(a, b);
        const bool inS = S[v] != 0;
        cut += (unsigned long long)(inS ? b : a);
        const int tc = st.tcap[v];
        if (tc < 0 || tc > b - m) ++bad;
        tin += (unsigned long long)(b - tc);
        long long e = (long long)(a - m) - (long long)(b - m - tc);
#pragma unroll
        for (int d = 0; d < arcs_of(CONN); ++d) {
            const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d), wz = z + arc_dz(CONN, d);
            const int r = st.cap[(size_t)d * n + v];
            if (!in_grid(g, wx, wy, wz)) {
                if (r != 0) ++bad;
                continue;
            }
            const size_t w = ((size_t)wz * g.Y + wy) * g.X + wx;
            const int c = (d & 1) ? nl[(size_t)(d >> 1) * n + w] : nl[(size_t)(d >> 1) * n + v];
            const int rr = st.cap[(size_t)(d ^ 1) * n + w];
            if (r < 0 || (long long)r + rr != 2ll * c) ++bad;
            e -= (long long)c - r;
            if (inS && !S[w]) cut += (unsigned long long)c;
        }
        if (e != st.exc[v] || e < 0) ++bad;
    }
    for (int o = 16; o > 0; o >>= 1) {
        cut += __shfl_down_sync(0xffffffffu, cut, o);
        tin += __shfl_down_sync(0xffffffffu, tin, o);
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (cut) atomicAdd(&sums[0], cut);
        if (tin) atomicAdd(&sums[1], tin);
        if (bad) atomicAdd(&sums[2], bad);
    }
}

template <int CONN>
static cudaError_t launch_certify(mf_grid *g, unsigned long long *sums) {
    // a solve on reduced inputs is certified on them (the merged vertices are
    // isolated there, so S_min with S* added has the same cut capacity)
    const int *cs = g->reduced ? g->red_cs : g->cs, *ct = g->reduced ? g->red_ct : g->ct;
    const int *nl = g->reduced ? g->red_nl : g->nl;
    certify_kernel<CONN><<<grid_blocks(g->g.n, 256), 256, 0, g->stream>>>(g->g, g->st, cs, ct, nl, g->smin, sums);
    return cudaGetLastError();
}

// |B| of Sec. 4.1 for a tiling: a vertex is a boundary vertex iff along some
// axis it is the first cell of a tile (not at 0) or the last (not at the end);
// the same set for 4- and 8-connectivity (diagonal neighbours in another tile
// imply a straight one) and for the 6-connected 3D stencil.
static long long boundary_count(const Geom &g) {
    auto inner = [](long long D, long long T) {
        long long b = 0;
        for (long long c = 0; c < D; ++c)
            if ((c % T == 0 && c > 0) || (c % T == T - 1 && c < D - 1)) ++b;
        return D - b;
    };
    return (long long)g.n - inner(g.X, g.tx) * inner(g.Y, g.ty) * inner(g.Z, g.tz);
}

// |B| for a stencil with longer displacements: the vertices with an in-grid
// neighbour in another region, counted on one tile position per class of
// tiles (interior tiles share one count, edge tiles are counted one by one)
static long long boundary_count_stencil(const Geom &g, int conn) {
    const int H = arcs_of(conn) / 2;
    long long b = 0;
    for (int ry = 0; ry < g.RY; ++ry)
        for (int rx = 0; rx < g.RX; ++rx) {
            const bool interior = rx > 0 && rx + 1 < g.RX && ry > 0 && ry + 1 < g.RY;
            if (interior && !(rx == 1 && ry == 1)) continue;  // counted once below
            long long c = 0;
            for (int ly = 0; ly < g.ty; ++ly)
                for (int lx = 0; lx < g.tx; ++lx) {
                    const int x = rx * g.tx + lx, y = ry * g.ty + ly;
                    if (x >= g.X || y >= g.Y) continue;
                    bool inB = false;
                    for (int d = 0; d < 2 * H && !inB; ++d) {
                        const int wx = x + ((d & 1) ? -paper_dx(d >> 1) : paper_dx(d >> 1));
                        const int wy = y + ((d & 1) ? -paper_dy(d >> 1) : paper_dy(d >> 1));
                        if (wx < 0 || wx >= g.X || wy < 0 || wy >= g.Y) continue;
                        inB = (wx >> g.sx) != rx || (wy >> g.sy) != ry;
                    }
                    c += inB;
                }
            b += interior ? c * (long long)(g.RX - 2) * (g.RY - 2) : c;
        }
    return b;
}

extern "C" {

void mf_default_opts(mf_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->max_sweeps = 0;
    o->partial_discharge = 0;
    o->global_gap = 1;
    o->global_relabel_period = 4;
    o->max_rounds = 0;
}

const char *mf_last_error(const mf_grid *g) { return g ? g->err.c_str() : g_static_err.c_str(); }

static void free_graph(mf_grid *h) {
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->graph_exec = nullptr;
    h->graph = nullptr;
}

static void free_all(mf_grid *h) {
    free_graph(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->loopctl) cudaFree(h->loopctl);
    if (h->h_loop) cudaFreeHost(h->h_loop);
    h->cap_stream = nullptr;
    h->loopctl = nullptr;
    h->h_loop = nullptr;
    void *planes[] = {h->cs, h->ct, h->nl, h->st.cap, h->st.tcap, h->st.exc, h->st.lab, h->st.lab_next, h->st.bout};
    for (void *p : planes)
        if (p) {
            if (h->host_state) cudaFreeHost(p);
            else cudaFree(p);
        }
    void *ptrs[] = {h->st.active, h->st.disc, h->st.left_active, h->st.flow_t, h->st.flow0,
                    h->st.hist, h->st.ctr, h->smin, h->tset, h->c64, h->cut_scratch, h->warmF, h->warmFt,
                    h->warmE};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->h_ctr) cudaFreeHost(h->h_ctr);
    if (h->h_fin) cudaFreeHost(h->h_fin);
    if (h->h_warm) cudaFreeHost(h->h_warm);
    for (void *p : {(void *)h->red_codes, (void *)h->red_cs, (void *)h->red_ct, (void *)h->red_nl, (void *)h->red_dev})
        if (p) cudaFree(p);
    if (h->h_red) cudaFreeHost(h->h_red);
    if (h->br_scratch) cudaFree(h->br_scratch);
    if (h->h_br) cudaFreeHost(h->h_br);
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

mf_status mf_create_grid(mf_grid **out, int ndim, const int64_t dims[3], int connectivity,
                         const int32_t tile[3], void *cuda_stream) {
    return mf_create_grid_ex(out, ndim, dims, connectivity, tile, cuda_stream, 0);
}

mf_status mf_create_grid_ex(mf_grid **out, int ndim, const int64_t dims[3], int connectivity,
                            const int32_t tile[3], void *cuda_stream, int flags) {
    mf_grid *g = nullptr;
    if (flags & ~MF_STATE_HOST) return fail(nullptr, MF_EINVAL, "unknown flags");
    if (!out) return fail(nullptr, MF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, MF_EINVAL, "dims is NULL");
    const bool paper = ndim == 2 && connectivity >= 108 && connectivity <= 128 && connectivity % 4 == 0;
    if (!((ndim == 2 && (connectivity == 4 || connectivity == 8)) || paper || (ndim == 3 && connectivity == 6)))
        return fail(nullptr, MF_EINVAL, "connectivity must be 4, 8 or MF_PAPER_STENCIL(8..28) (ndim 2) or 6 (ndim 3)");
    if (paper && (flags & MF_STATE_HOST)) return fail(nullptr, MF_EINVAL, "MF_STATE_HOST is for the 4/8/6 stencils");
    long long X = dims[0], Y = dims[1], Z = ndim == 3 ? dims[2] : 1;
    if (X < 1 || Y < 1 || Z < 1 || X > INT_MAX || Y > INT_MAX || Z > INT_MAX)
        return fail(nullptr, MF_EINVAL, "dims must be >= 1");
    long long nll = X * Y * Z;
    if (nll > (1ll << 31) - 1) return fail(nullptr, MF_EINVAL, "more than 2^31-1 vertices");
    int tx = 32, ty = 32, tz = 1;
    if (ndim == 3) { tx = 32; ty = 8; tz = 4; }
    if (tile && (tile[0] | tile[1] | tile[2])) {
        tx = tile[0];
        ty = tile[1];
        tz = ndim == 3 ? tile[2] : 1;
    }
    if (!discharge_supported(connectivity, tx, ty, tz))
        return fail(nullptr, MF_EINVAL, "unsupported tile shape for this connectivity");
    g = new (std::nothrow) mf_grid();
    if (!g) return fail(nullptr, MF_ENOMEM, "host allocation failed");
    g->ndim = ndim;
    g->host_state = (flags & MF_STATE_HOST) != 0;
    g->st.host = g->host_state ? 1 : 0;
    g->conn = connectivity;
    g->H = arcs_of(connectivity) / 2;
    g->N = arcs_of(connectivity);
    Geom &G = g->g;
    G.X = (int)X; G.Y = (int)Y; G.Z = (int)Z; G.n = nll;
    G.tx = tx; G.ty = ty; G.tz = tz;
    G.sx = __builtin_ctz(tx); G.sy = __builtin_ctz(ty); G.sz = __builtin_ctz(tz);
    G.RX = (int)((X + tx - 1) / tx); G.RY = (int)((Y + ty - 1) / ty); G.RZ = (int)((Z + tz - 1) / tz);
    G.nreg = G.RX * G.RY * G.RZ;
    g->boundary = paper ? boundary_count_stencil(G, connectivity) : boundary_count(G);
    G.dinf = (int)std::max<long long>(g->boundary, 1);
    auto bail = [&](mf_status s) { free_all(g); std::string m = g->err; delete g; g_static_err = m; return s; };
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) { g->err = std::string("no CUDA device: ") + cudaGetErrorString(e); return bail(MF_ECUDA); }
    if (cuda_stream) {
        g->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MF_ECUDA); }
        g->own_stream = true;
    }
    const size_t N = (size_t)arcs_of(connectivity);
    const size_t n = (size_t)nll;
    // the planes and stored inputs: device memory, or with MF_STATE_HOST pinned
    // host memory that the kernels read and write over NVLink-C2C
    struct A { void **p; size_t bytes; } planes[] = {
        {(void **)&g->cs, n * 4}, {(void **)&g->ct, n * 4}, {(void **)&g->nl, (N / 2) * n * 4},
        {(void **)&g->st.cap, N * n * 4}, {(void **)&g->st.tcap, n * 4}, {(void **)&g->st.exc, n * 4},
        {(void **)&g->st.lab, n * 4}, {(void **)&g->st.lab_next, n * 4}, {(void **)&g->st.bout, N * n * 4}};
    for (auto &a : planes) {
        e = g->host_state ? cudaMallocHost(a.p, a.bytes) : cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            g->err = std::string(g->host_state ? "cudaMallocHost: " : "cudaMalloc: ") + cudaGetErrorString(e);
            return bail(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA);
        }
    }
    A allocs[] = {
        {(void **)&g->st.active, (size_t)G.nreg}, {(void **)&g->st.disc, (size_t)G.nreg},
        {(void **)&g->st.left_active, (size_t)G.nreg}, {(void **)&g->st.flow_t, 8}, {(void **)&g->st.flow0, 8},
        {(void **)&g->st.hist, (kHistBins + 1) * 4}, {(void **)&g->st.ctr, kCtrWords * 4},
        {(void **)&g->smin, (size_t)n}, {(void **)&g->tset, (size_t)n}, {(void **)&g->c64, sizeof(Counters64)},
        {(void **)&g->cut_scratch, paper ? stencil_glr_scratch_bytes(G) : ndim == 2 ? cut2d_scratch_bytes(G, connectivity)
                                                       : (glr3d_supported(G) ? glr3d_scratch_bytes(G) : 0)}};
    for (auto &a : allocs) {
        if (a.bytes == 0) continue;
        e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            g->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            return bail(e == cudaErrorMemoryAllocation ? MF_ENOMEM : MF_ECUDA);
        }
    }
    e = cudaMallocHost((void **)&g->h_ctr, kCtrWords * 4);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_fin, sizeof(mf_grid::FinishHost));
    if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MF_ENOMEM); }
    g->h_ctr_dv = (int *)device_view(g->h_ctr);
    g->h_fin_dv = (mf_grid::FinishHost *)device_view(g->h_fin);
    if (!g->h_ctr_dv || !g->h_fin_dv) { g->err = "pinned host memory without a device view"; return bail(MF_ECUDA); }
    for (auto &ev : g->ev) {
        e = cudaEventCreate(&ev);
        if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MF_ECUDA); }
    }
    e = cudaMemsetAsync(g->st.disc, 0, (size_t)G.nreg, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->st.left_active, 0, (size_t)G.nreg, g->stream);
    if (e == cudaSuccess && !g->host_state) e = cudaMemsetAsync(g->st.bout, 0, N * n * 4, g->stream);
    if (e != cudaSuccess) { g->err = cudaGetErrorString(e); return bail(MF_ECUDA); }
    if (g->host_state) memset(g->st.bout, 0, N * n * 4);
    mf_default_opts(&g->opts);
    *out = g;
    return MF_OK;
}

mf_status mf_destroy(mf_grid *g) {
    if (!g) return MF_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    free_all(g);
    delete g;
    return MF_OK;
}

// mf_set_caps in phases: the copies, the validation kernel, the read-back of
// its flags (each enqueued on the grid's stream), then (after a wait) the
// status.  A batch runs each phase for all grids before the next, so that
// the copies follow one another on the copy engine instead of alternating
// with the validation kernels.
static mf_status set_caps_copies(mf_grid *g, const int32_t *cs, const int32_t *ct, const int32_t *nlink) {
    if (!cs || !ct || !nlink) return fail(g, MF_EINVAL, "cs, ct and nlink must be non-NULL");
    const size_t n = (size_t)g->g.n, H = (size_t)g->H;
    g->caps_set = false;
    g->begun = g->finished = false;
    g->flow_cached = false;
    g->warm_ready = false;
    const cudaMemcpyKind kind = cudaMemcpyDefault;  // unified addressing: the direction follows from the pointers
    CK(cudaMemcpyAsync(g->cs, cs, n * 4, kind, g->stream));
    CK(cudaMemcpyAsync(g->ct, ct, n * 4, kind, g->stream));
    CK(cudaMemcpyAsync(g->nl, nlink, H * n * 4, kind, g->stream));
    return MF_OK;
}
static mf_status set_caps_validate(mf_grid *g) {
    CK(cudaMemsetAsync(g->st.ctr, 0, kCtrWords * 4, g->stream));
    CK(DISPATCH(g->conn, launch_validate, g, &g->st.ctr[kError]));
    return MF_OK;
}
static mf_status set_caps_readback(mf_grid *g) {
    CK(cudaMemcpyAsync(g->h_ctr, g->st.ctr, kCtrWords * 4, cudaMemcpyDeviceToHost, g->stream));
    return MF_OK;
}
static mf_status set_caps_enqueue(mf_grid *g, const int32_t *cs, const int32_t *ct, const int32_t *nlink) {
    mf_status st = set_caps_copies(g, cs, ct, nlink);
    if (st == MF_OK) st = set_caps_validate(g);
    if (st == MF_OK) st = set_caps_readback(g);
    return st;
}
static mf_status set_caps_status(mf_grid *g) {
    const int f = g->h_ctr[kError];
    if (f & 1) return fail(g, MF_EINVAL, "negative capacity");
    if (f & 2) return fail(g, MF_EINVAL, "nonzero neighbour capacity leaving the grid");
    if (f & 4) return fail(g, MF_EOVERFLOW, "capacities could overflow int32");
    g->caps_set = true;
    return MF_OK;
}

mf_status mf_set_caps(mf_grid *g, const int32_t *cs, const int32_t *ct, const int32_t *nlink, int on_device) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    (void)on_device;
    mf_status st = set_caps_enqueue(g, cs, ct, nlink);
    if (st != MF_OK) return st;
    CK(cudaStreamSynchronize(g->stream));
    return set_caps_status(g);
}

// one wait per distinct stream of the grids
static cudaError_t sync_streams(mf_grid *const *grids, int count) {
    std::vector<cudaStream_t> done;
    for (int i = 0; i < count; ++i) {
        const cudaStream_t s = grids[i]->stream;
        if (std::find(done.begin(), done.end(), s) != done.end()) continue;
        done.push_back(s);
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// one launch copies many segments (src and dst device-accessible: device or
// pinned host memory, read over NVLink-C2C); 16-byte words where both ends
// and the length allow, 4-byte words otherwise
struct CopySeg {
    const void *src;
    void *dst;
    unsigned long long bytes;
};
__global__ void gather_copy_kernel(const CopySeg *__restrict__ segs, int nseg) {
    for (int k = blockIdx.y; k < nseg; k += gridDim.y) {
        const CopySeg sg = segs[k];
        const bool v16 = ((reinterpret_cast<uintptr_t>(sg.src) | reinterpret_cast<uintptr_t>(sg.dst) | sg.bytes) & 15) == 0;
        const size_t stride = (size_t)gridDim.x * blockDim.x;
        if (v16) {
            const int4 *a = (const int4 *)sg.src;
            int4 *b = (int4 *)sg.dst;
            for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sg.bytes / 16; i += stride) b[i] = a[i];
        } else {
            const int *a = (const int *)sg.src;
            int *b = (int *)sg.dst;
            for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < sg.bytes / 4; i += stride) b[i] = a[i];
        }
    }
}

mf_status mf_set_caps_batch(mf_grid *const *grids, int count, const int32_t *const *cs, const int32_t *const *ct,
                            const int32_t *const *nlink, int on_device) {
    mf_grid *g = nullptr;
    (void)on_device;
    if (!grids || count < 1 || !cs || !ct || !nlink) return fail(nullptr, MF_EINVAL, "bad batch arguments");
    for (int i = 0; i < count; ++i)
        if (!grids[i]) return fail(nullptr, MF_EINVAL, "null grid in the batch");
    g = grids[0];
    for (int i = 0; i < count; ++i)
        if (!cs[i] || !ct[i] || !nlink[i]) return fail(g, MF_EINVAL, std::string("grid ") + std::to_string(i) +
                                                                  ": cs, ct and nlink must be non-NULL");
    // on one stream, with sources a kernel can read: one gather launch for all
    // copies (a copy per array costs more than its bytes on small grids)
    bool gather = true;
    std::vector<const void *> views((size_t)count * 3, nullptr);
    for (int i = 0; i < count && gather; ++i) {
        views[3 * i] = device_view(cs[i]);
        views[3 * i + 1] = device_view(ct[i]);
        views[3 * i + 2] = device_view(nlink[i]);
        gather = grids[i]->stream == g->stream && views[3 * i] && views[3 * i + 1] && views[3 * i + 2];
    }
    if (gather) {
        std::vector<CopySeg> segs;
        segs.reserve((size_t)count * 3);
        for (int i = 0; i < count; ++i) {
            mf_grid *h = grids[i];
            const unsigned long long n4 = (unsigned long long)h->g.n * 4;
            segs.push_back({views[3 * i], h->cs, n4});
            segs.push_back({views[3 * i + 1], h->ct, n4});
            segs.push_back({views[3 * i + 2], h->nl, (unsigned long long)h->H * n4});
            h->caps_set = false;
            h->begun = h->finished = false;
            h->flow_cached = false;
            h->warm_ready = false;
        }
        CopySeg *dsegs = nullptr;
        CK(cudaMallocAsync((void **)&dsegs, segs.size() * sizeof(CopySeg), g->stream));
        CK(cudaMemcpyAsync(dsegs, segs.data(), segs.size() * sizeof(CopySeg), cudaMemcpyHostToDevice, g->stream));
        const int ns = (int)segs.size();
        gather_copy_kernel<<<dim3(64, std::min(ns, 65535)), 256, 0, g->stream>>>(dsegs, ns);
        CK(cudaGetLastError());
        CK(cudaFreeAsync(dsegs, g->stream));
        bool unit_stencils = true;  // the batched validation covers the 4/8/6 stencils
        for (int i = 0; i < count; ++i) unit_stencils &= !is_paper(grids[i]->conn);
        if (unit_stencils) {
            // every grid's validation in one launch, one read-back of the flags
            std::vector<ValJob> jobs((size_t)count);
            std::vector<int2> units;
            for (int i = 0; i < count; ++i) {
                mf_grid *h = grids[i];
                jobs[i] = ValJob{h->g, h->cs, h->ct, h->nl, h->conn};
                const long long nc = (h->g.n + kValChunk - 1) / kValChunk;
                for (long long c = 0; c < nc; ++c) units.push_back(make_int2(i, (int)c));
            }
            ValJob *djobs = nullptr;
            int2 *dunits = nullptr;
            int *dflags = nullptr;
            std::vector<int> hflags((size_t)count, 0);
            CK(cudaMallocAsync((void **)&djobs, jobs.size() * sizeof(ValJob), g->stream));
            CK(cudaMallocAsync((void **)&dunits, units.size() * sizeof(int2), g->stream));
            CK(cudaMallocAsync((void **)&dflags, (size_t)count * sizeof(int), g->stream));
            CK(cudaMemcpyAsync(djobs, jobs.data(), jobs.size() * sizeof(ValJob), cudaMemcpyHostToDevice, g->stream));
            CK(cudaMemcpyAsync(dunits, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice, g->stream));
            CK(cudaMemsetAsync(dflags, 0, (size_t)count * sizeof(int), g->stream));
            const int nu = (int)units.size();
            validate_batch_kernel<<<std::min(nu, device_sms() * 16), 256, 0, g->stream>>>(djobs, dunits, nu, dflags);
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(hflags.data(), dflags, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, g->stream));
            CK(cudaFreeAsync(djobs, g->stream));
            CK(cudaFreeAsync(dunits, g->stream));
            CK(cudaFreeAsync(dflags, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            for (int i = 0; i < count; ++i) {
                grids[i]->h_ctr[kError] = hflags[i];
                mf_status st = set_caps_status(grids[i]);
                if (st != MF_OK) {
                    if (grids[i] != g) fail(g, st, std::string("grid ") + std::to_string(i) + ": " + grids[i]->err);
                    return st;
                }
            }
            return MF_OK;
        }
    }
    for (int phase = gather ? 1 : 0; phase < 3; ++phase)
        for (int i = 0; i < count; ++i) {
            mf_status st = phase == 0 ? set_caps_copies(grids[i], cs[i], ct[i], nlink[i])
                           : phase == 1 ? set_caps_validate(grids[i]) : set_caps_readback(grids[i]);
            if (st != MF_OK) {
                if (grids[i] != g) fail(g, st, std::string("grid ") + std::to_string(i) + ": " + grids[i]->err);
                return st;
            }
        }
    CK(sync_streams(grids, count));
    for (int i = 0; i < count; ++i) {
        mf_status st = set_caps_status(grids[i]);
        if (st != MF_OK) {
            if (grids[i] != g) fail(g, st, std::string("grid ") + std::to_string(i) + ": " + grids[i]->err);
            return st;
        }
    }
    return MF_OK;
}

// The region reduction of Sec. 8 on the stored inputs: class codes of every
// vertex into g->red_codes (and the reduced-input buffers allocated); the
// counts and the round-cap flag are read back (one wait).  *ok = false if an
// Augment of some region hit the round cap (the codes are then not used).
static mf_status reduction_run(mf_grid *g, const int32_t *tile, bool *ok) {
    int t[3] = {g->g.tx, g->g.ty, g->g.tz};
    if (tile && (tile[0] | tile[1] | tile[2])) {
        t[0] = tile[0];
        t[1] = tile[1];
        t[2] = g->ndim == 3 ? tile[2] : 1;
    }
    RedGeom rg{};
    if (!reduction_supported(g->conn, t, &rg, g->g)) {
        // the solver's tile does not fit one region network into shared memory
        if (tile && (tile[0] | tile[1] | tile[2])) return fail(g, MF_EINVAL, "reduction tile too large");
        const int d2[3] = {32, 32, 1}, d3[3] = {32, 8, 4};
        if (!reduction_supported(g->conn, g->ndim == 3 ? d3 : d2, &rg, g->g))
            return fail(g, MF_EINVAL, "no supported reduction tile");
    }
    const size_t n = (size_t)g->g.n;
    if (!g->red_codes) {
        CK(cudaMalloc(&g->red_codes, n));
        CK(cudaMalloc(&g->red_cs, n * 4));
        CK(cudaMalloc(&g->red_ct, n * 4));
        CK(cudaMalloc(&g->red_nl, (size_t)g->H * n * 4));
        CK(cudaMalloc(&g->red_dev, 8 * sizeof(unsigned long long)));
        CK(cudaMallocHost((void **)&g->h_red, 8 * sizeof(unsigned long long)));
    }
    CK(cudaMemsetAsync(g->red_dev, 0, 8 * sizeof(unsigned long long), g->stream));
    const int mr = g->opts.max_rounds > 0 ? g->opts.max_rounds : 1 << 16;
    CK(launch_region_reduction(g->conn, rg, g->cs, g->ct, g->nl, g->red_codes, g->red_dev, mr, (int *)&g->red_dev[5],
                               g->stream));
    // red_dev[4] (zero here) later receives the constant of the merged inputs
    CK(cudaMemcpyAsync(g->h_red, g->red_dev, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    *ok = ((int *)&g->h_red[5])[0] == 0;
    return MF_OK;
}

// counts of the relabel of a warm mf_begin, after the stream has been waited for
static void begin_collect(mf_grid *g) {
    if (!g->begin_pending) return;
    g->begin_active = g->h_ctr[kActiveRegions];
    g->stats.relabel_levels = g->h_ctr[kGlrLevels];
    g->begin_pending = false;
}

// defer: leave the relabel of a warm start in flight (a batch waits once for
// all its grids and then calls begin_collect)
static mf_status begin_impl(mf_grid *g, const mf_opts *opts, bool defer, bool *batched_init = nullptr);

mf_status mf_begin(mf_grid *g, const mf_opts *opts) { return begin_impl(g, opts, false); }

// batched_init: a cold start without region reduction leaves its device
// reset and Init to the caller (set to true then), who runs them for many
// grids at once
static mf_status begin_impl(mf_grid *g, const mf_opts *opts, bool defer, bool *batched_init) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!g->caps_set) return fail(g, MF_ESTATE, "mf_set_caps has not succeeded");
    if (opts) g->opts = *opts;
    else mf_default_opts(&g->opts);
    if (g->opts.max_rounds <= 0) g->opts.max_rounds = 1 << 16;
    if (g->opts.kernel_variant < 0 || g->opts.kernel_variant > 2) return fail(g, MF_EINVAL, "kernel_variant must be 0, 1 or 2");
    if (is_paper(g->conn) && (g->opts.warm_start || g->opts.region_reduction || g->opts.boundary_relabel_period > 0))
        return fail(g, MF_EINVAL, "the Sec. 7.1 stencils run without warm start, region reduction and boundary relabel");
    // Discharge = PRD (kernel_variant 2): distance labels with unit arc lengths
    // reach up to n - 1, so d_inf = n; the global gap on boundary labels relies
    // on ARD's region distances (labels drop only between regions) and is off
    if (g->opts.kernel_variant == 2) {
        if (g->opts.warm_start || g->opts.region_reduction)
            return fail(g, MF_EINVAL, "the PRD discharge runs cold and unreduced");
        g->g.dinf = (int)std::max<long long>(g->g.n, 1);
        g->opts.global_gap = 0;
    } else {
        g->g.dinf = (int)std::max<long long>(g->boundary, 1);
    }
    const size_t nreg = (size_t)g->g.nreg;
    const bool defer_init = batched_init && !g->opts.warm_start && !g->opts.region_reduction;
    if (batched_init) *batched_init = defer_init;
    if (defer_init) {  // the caller resets the state and runs Init
        g->reduced = false;
        g->launches = 0;
        g->sweep = 0;
        g->begun = true;
        g->finished = false;
        g->flow_cached = false;
        memset(&g->stats, 0, sizeof(g->stats));
        g->stats.boundary_size = (int32_t)g->boundary;
        g->begin_active = -1;
        return MF_OK;
    }
    CK(cudaMemsetAsync(g->st.active, 0, nreg, g->stream));
    CK(cudaMemsetAsync(g->st.disc, 0, nreg, g->stream));
    CK(cudaMemsetAsync(g->st.left_active, 0, nreg, g->stream));
    CK(cudaMemsetAsync(g->st.flow_t, 0, 8, g->stream));
    CK(cudaMemsetAsync(g->st.flow0, 0, 8, g->stream));
    CK(cudaMemsetAsync(g->st.ctr, 0, kCtrWords * 4, g->stream));
    CK(cudaMemsetAsync(g->c64, 0, sizeof(Counters64), g->stream));
    CK(cudaMemsetAsync(g->st.hist, 0, (kHistBins + 1) * 4, g->stream));
    g->reduced = false;
    int red_launches = 0;
    if (g->opts.region_reduction) {
        if (g->opts.warm_start) return fail(g, MF_EINVAL, "region_reduction and warm_start cannot be combined");
        bool ok = false;
        mf_status rs = reduction_run(g, nullptr, &ok);
        if (rs != MF_OK) return rs;
        if (ok) {
            // merge S* into s and T* into t: reduced inputs, the constant into flow0
            CK(launch_reduction_apply(g->conn, g->g, g->red_codes, g->cs, g->ct, g->nl, g->red_cs, g->red_ct,
                                      g->red_nl, (unsigned long long *)g->st.flow0, &g->red_dev[4], g->stream));
            CK(cudaMemcpyAsync(&g->h_red[4], &g->red_dev[4], 8, cudaMemcpyDeviceToHost, g->stream));
            g->reduced = true;
            red_launches = 2;
        }
    }
    if (g->opts.warm_start) {
        if (!g->warm_ready) return fail(g, MF_ESTATE, "warm_start requested without a successful mf_warm_start");
        CK(launch_warm_init(g->conn, g->g, g->st, g->cs, g->ct, g->nl, g->warmF, g->warmFt, g->warmE, g->stream));
    } else {
        CK(DISPATCH(g->conn, launch_init, g));
    }
    hist_init_kernel<<<1, 32, 0, g->stream>>>(g->st, (int)g->boundary);
    CK(cudaGetLastError());
    g->launches = 2 + red_launches;
    g->sweep = 0;
    g->begun = true;
    g->finished = false;
    g->flow_cached = false;
    memset(&g->stats, 0, sizeof(g->stats));
    g->stats.boundary_size = (int32_t)g->boundary;
    g->stats.projection_rounds = g->opts.warm_start ? g->warm_rounds : 0;
    g->stats.reduced_vertices = g->reduced ? (int32_t)(g->h_red[0] + g->h_red[1]) : 0;
    g->begin_active = -1;
    if (g->opts.warm_start && g->ndim == 2 && glr2d_supported(g->g)) {
        // A projected preflow leaves excess where the prediction was wrong and
        // labels 0 everywhere; exact region distances (a valid labeling) put the
        // excess that cannot reach t at d-infinity before the first sweep, so
        // the sweeps only move the excess that still can.
        CK(glr2d(g->conn, g->g, g->st, g->cut_scratch, g->stream));
        CK(cudaMemcpyAsync(g->h_ctr, g->st.ctr, kCtrWords * 4, cudaMemcpyDeviceToHost, g->stream));
        g->begin_pending = true;
        g->stats.global_relabels = 1;
        g->launches += 4;  // masks, the cooperative levels launch, finish, count
        if (!defer) {
            CK(cudaStreamSynchronize(g->stream));
            begin_collect(g);
        }
    }
    return MF_OK;
}

// the global relabel (exact region distance), 2D or 3D
static bool glr_supported(const mf_grid *g) {
    if (is_paper(g->conn)) return stencil_glr_supported(g->conn, g->g);  // the bit-mask relabels take unit steps only
    return g->ndim == 2 ? glr2d_supported(g->g) : glr3d_supported(g->g);
}
// (enqueued without waiting; the levels run are left in st.ctr[kGlrLevels])
static cudaError_t glr_run(mf_grid *g, cudaStream_t s) {
    if (is_paper(g->conn)) return stencil_glr(g->conn, g->g, g->st, g->cut_scratch, s);
    return g->ndim == 2 ? glr2d(g->conn, g->g, g->st, g->cut_scratch, s) : glr3d(g->g, g->st, g->cut_scratch, s);
}

// which relabel (if any) follows sweep count s: the exact global relabel
// where its period divides s, else the boundary relabel where its period does
static bool glr_due(const mf_grid *g, int s) {
    const int P = g->opts.global_relabel_period, F = g->opts.global_relabel_first;
    return ((P > 0 && s % P == 0) || (F > 0 && s == F)) && glr_supported(g);
}
static bool br_due(const mf_grid *g, int s) {
    const int P = g->opts.boundary_relabel_period;
    return P > 0 && s % P == 0 && !glr_due(g, s);
}
// the graph loops stop where either relabel may be due
static int relabel_stop_period(const mf_opts &o, bool glr_ok) {
    const int a = glr_ok ? std::max(0, o.global_relabel_period) : 0, b = std::max(0, o.boundary_relabel_period);
    if (!a) return b;
    if (!b) return a;
    int x = a, y = b;
    while (y) { const int t = x % y; x = y; y = t; }
    return x;
}

// one boundary relabel (Sec. 6.1) on g's stream; *active = regions active after it
static mf_status br_step(mf_grid *g, cudaStream_t s, int *active, BrResult *r) {
    if (!g->br_scratch) {
        CK(cudaMalloc(&g->br_scratch, br_scratch_bytes(g->g, g->conn)));
        CK(cudaMallocHost((void **)&g->h_br, 8 * 4));
    }
    BrResult res{};
    CK(boundary_relabel(g->conn, g->g, g->st, g->br_scratch, g->h_br, &res, s));
    g->launches += res.launches;
    if (res.applied) {
        g->stats.boundary_relabels++;
        g->stats.boundary_relabel_levels += res.levels;
    }
    if (active) {
        CK(cudaMemcpyAsync(g->h_ctr, g->st.ctr, kCtrWords * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *active = g->h_ctr[kActiveRegions];
    }
    if (r) *r = res;
    return MF_OK;
}

static mf_status run_sweep(mf_grid *g, int32_t *active_out) {
    g->flow_cached = false;
    SweepArgs sa{};
    sa.sweep = g->sweep;
    sa.partial = g->opts.partial_discharge;
    sa.max_rounds = g->opts.max_rounds;
    sa.variant = g->opts.kernel_variant;
    sa.c64 = g->c64;
    CK(cudaMemsetAsync(g->st.ctr, 0, 4 * (kGap + 1), g->stream));  // active count, error, gap
    CK(cudaEventRecord(g->ev[4], g->stream));
    CK(launch_discharge(g->conn, g->g, g->st, sa, g->stream));
    CK(cudaEventRecord(g->ev[5], g->stream));
    CK(DISPATCH(g->conn, launch_fuse_post, g, g->opts.global_gap != 0, g->stream));
    CK(cudaEventRecord(g->ev[6], g->stream));
    g->launches += g->opts.global_gap ? 5 : 4;
    CK(cudaMemcpyAsync(g->h_ctr, g->st.ctr, kCtrWords * 4, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    {
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, g->ev[4], g->ev[5]);
        cudaEventElapsedTime(&b, g->ev[5], g->ev[6]);
        g->stats.ms_discharge += a;
        g->stats.ms_fuse += b;
        g->stats.discharge_launches++;
    }
    ++g->sweep;
    g->stats.sweeps = g->sweep;
    if (g->h_ctr[kGap] > 0) g->stats.gaps++;
    if (g->h_ctr[kError]) {
        if (active_out) *active_out = g->h_ctr[kActiveRegions];
        if (g->h_ctr[kError] == 2) return fail(g, MF_ECUDA, "a bulk copy into shared memory did not complete");
        return fail(g, MF_EROUNDLIMIT, "an Augment stage hit max_rounds");
    }
    int active = g->h_ctr[kActiveRegions];
    const bool relabel = active > 0 && (glr_due(g, g->sweep) || br_due(g, g->sweep));
    if (relabel) CK(cudaEventRecord(g->ev[7], g->stream));
    if (active > 0 && glr_due(g, g->sweep)) {
        // exact region-distance relabel (raises labels to max(d, d*)), then the
        // activity of every region is recomputed from the new labels
        CK(glr_run(g, g->stream));
        CK(cudaMemcpyAsync(g->h_ctr, g->st.ctr, kCtrWords * 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        const int levels = g->h_ctr[kGlrLevels];
        active = g->h_ctr[kActiveRegions];
        g->stats.global_relabels++;
        g->stats.relabel_levels += levels;
        g->launches += 4;  // masks, the cooperative levels launch, finish, count
    } else if (active > 0 && br_due(g, g->sweep)) {
        mf_status bs = br_step(g, g->stream, &active, nullptr);
        if (bs != MF_OK) return bs;
    }
    if (relabel) {  // both relabels end with a wait on the stream
        CK(cudaEventRecord(g->ev[8], g->stream));
        CK(cudaEventSynchronize(g->ev[8]));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev[7], g->ev[8]);
        g->stats.ms_relabel += ms;
    }
    if (active_out) *active_out = active;
    return MF_OK;
}

mf_status mf_sweep(mf_grid *g, int32_t *active) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!g->begun) return fail(g, MF_ESTATE, "mf_begin has not been called");
    return run_sweep(g, active);
}

mf_status mf_boundary_relabel(mf_grid *g, int32_t *info) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!g->begun) return fail(g, MF_ESTATE, "mf_begin has not been called");
    int active = 0;
    BrResult r{};
    mf_status s = br_step(g, g->stream, &active, &r);
    if (s != MF_OK) return s;
    if (info) {
        info[0] = active;
        info[1] = r.levels;
        info[2] = r.merged;
        info[3] = r.applied;
    }
    return MF_OK;
}

// The cut extraction and the read-back of the flow value and counters,
// enqueued on stream st without waiting (results land in g->h_fin); the
// closures of 2D grids and of 3D grids with 32-wide tiles run on the device
// to their fixed point, other 3D tiles loop on the host.
// copies = false: the caller has the flow parts and stage counts read back
static mf_status finish_enqueue(mf_grid *g, cudaStream_t st, bool cut_done = false, bool copies = true) {
    if (!cut_done) g->h_fin->passes[0] = g->h_fin->passes[1] = 0;
    if (cut_done) {
        // the cut closures ran batched with other grids
    } else if (g->ndim == 2 && !is_paper(g->conn)) {
        CK(cut2d(g->conn, g->g, g->st, g->cut_scratch, g->smin, g->tset, g->h_fin->passes, st));
        g->launches += 5;
    } else if (glr3d_supported(g->g)) {
        CK(cut3d(g->g, g->st, g->cut_scratch, g->smin, g->tset, g->h_fin->passes, st));
        g->launches += 5;
    } else {
        int passes = 0;
        cut_seed_kernel<<<grid_blocks(g->g.n, 256), 256, 0, st>>>(g->g, g->st, g->smin, g->tset);
        CK(cudaGetLastError());
        for (int which = 0; which < 2; ++which) {
            for (;;) {
                CK(cudaMemsetAsync(&g->st.ctr[kChanged], 0, 4, st));
                CK(DISPATCH(g->conn, launch_cut_pass, g, which == 0 ? g->smin : g->tset, which == 0 ? 1 : 0, st));
                ++g->launches;
                CK(cudaMemcpyAsync(g->h_ctr, g->st.ctr, kCtrWords * 4, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                ++passes;
                if (!g->h_ctr[kChanged]) break;
            }
        }
        complement_kernel<<<grid_blocks(g->g.n, 256), 256, 0, st>>>(g->tset, (size_t)g->g.n);
        CK(cudaGetLastError());
        g->launches += 2;
        g->h_fin->passes[0] = passes;
    }
    if (g->reduced) {  // S_min gains the strong sources, S_max loses the strong sinks
        CK(launch_reduction_cut((size_t)g->g.n, g->red_codes, g->smin, g->tset, st));
        ++g->launches;
    }
    if (!copies) return MF_OK;
    CK(cudaMemcpyAsync(&g->h_fin->f0, g->st.flow0, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&g->h_fin->ft, g->st.flow_t, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&g->h_fin->c, g->c64, sizeof(Counters64), cudaMemcpyDeviceToHost, st));
    return MF_OK;
}

// after the stream of finish_enqueue has been synchronised
static void finish_collect(mf_grid *g) {
    const mf_grid::FinishHost &f = *g->h_fin;
    g->stats.cut_passes = f.passes[0] + f.passes[1];
    g->stats.flow_value = f.f0 + (long long)f.ft;
    g->stats.stages = (int64_t)f.c.stages;
    g->stats.rounds = (int64_t)f.c.rounds;
    g->stats.discharges = (int64_t)f.c.discharges;
    g->stats.discharged_vertices = (int64_t)f.c.discharged_vertices;
    g->stats.launches = g->launches;
    g->red_konst = g->reduced ? (long long)g->h_red[4] : 0;
    g->finished = true;
    g->flow_cached = true;
}

mf_status mf_finish(mf_grid *g) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!g->begun) return fail(g, MF_ESTATE, "mf_begin has not been called");
    mf_status s = finish_enqueue(g, g->stream);
    if (s != MF_OK) return s;
    CK(cudaStreamSynchronize(g->stream));
    finish_collect(g);
    return MF_OK;
}

// Capture one sweep (counter reset, discharge, fusion, gap, activity, loop
// control) as the body of a while node, on a private stream (the caller's
// may be the legacy default stream, which cannot be captured).  Rebuilt when
// an option baked into the kernels' arguments changes.
static mf_status build_graph(mf_grid *g) {
    const int key[5] = {g->opts.partial_discharge, g->opts.max_rounds, g->opts.kernel_variant,
                        g->opts.global_gap != 0, 1};
    if (g->graph_exec && memcmp(key, g->graph_key, sizeof(key)) == 0) return MF_OK;
    free_graph(g);
    if (!g->cap_stream) CK(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    if (!g->loopctl) {
        CK(cudaMalloc(&g->loopctl, kLoopWords * 4));
        CK(cudaMallocHost((void **)&g->h_loop, kLoopWords * 4));
    }
    CK(cudaGraphCreate(&g->graph, 0));
    cudaGraphConditionalHandle handle;
    CK(cudaGraphConditionalHandleCreate(&handle, g->graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g->graph, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    SweepArgs sa{};
    sa.sweep_dev = &g->loopctl[kLoopSweep];
    sa.partial = g->opts.partial_discharge;
    sa.max_rounds = g->opts.max_rounds;
    sa.variant = g->opts.kernel_variant;
    sa.c64 = g->c64;
    cudaStream_t cs = g->cap_stream;
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaMemsetAsync(g->st.ctr, 0, 4 * (kGap + 1), cs);
    if (e == cudaSuccess) e = launch_discharge(g->conn, g->g, g->st, sa, cs);
    if (e == cudaSuccess) e = DISPATCH(g->conn, launch_fuse_post, g, g->opts.global_gap != 0, cs);
    if (e == cudaSuccess) {
        loop_ctl_kernel<<<1, 32, 0, cs>>>(g->st.ctr, g->loopctl, handle);
        e = cudaGetLastError();
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        free_graph(g);
        return fail(g, MF_ECUDA, std::string("sweep graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    CK(cudaGraphInstantiate(&g->graph_exec, g->graph, 0));
    memcpy(g->graph_key, key, sizeof(key));
    return MF_OK;
}

// The sweep loop on the device: the graph runs sweeps until no region is
// active, an error, the cap, or a multiple of the global-relabel period (the
// host then relabels and relaunches).  One host synchronisation per launch.
static mf_status run_graph_loop(mf_grid *g, long long cap) {
    mf_status s = build_graph(g);
    if (s != MF_OK) return s;
    const int P = relabel_stop_period(g->opts, glr_supported(g));
    int init[kLoopWords] = {0};
    init[kLoopSweep] = g->sweep;
    init[kLoopCap] = (int)std::min<long long>(cap, INT_MAX);
    init[kLoopPeriod] = P;
    init[kLoopFirst] = glr_supported(g) ? std::max(0, g->opts.global_relabel_first) : 0;
    memcpy(g->h_loop, init, sizeof(init));
    CK(cudaMemcpyAsync(g->loopctl, g->h_loop, kLoopWords * 4, cudaMemcpyHostToDevice, g->stream));
    const int per_sweep = g->opts.global_gap ? 6 : 5;
    for (;;) {
        const int before = g->sweep;
        CK(cudaGraphLaunch(g->graph_exec, g->stream));
        CK(cudaMemcpyAsync(g->h_loop, g->loopctl, kLoopWords * 4, cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        g->sweep = g->h_loop[kLoopSweep];
        g->launches += (g->sweep - before) * per_sweep;
        g->stats.sweeps = g->sweep;
        g->stats.gaps = g->h_loop[kLoopGaps];
        if (g->h_loop[kLoopError] == 2) return fail(g, MF_ECUDA, "a bulk copy into shared memory did not complete");
        if (g->h_loop[kLoopError]) return fail(g, MF_EROUNDLIMIT, "an Augment stage hit max_rounds");
        int active = g->h_loop[kLoopActive];
        if (active == 0) return MF_OK;
        if (g->sweep >= cap) return fail(g, MF_ESWEEPLIMIT, "sweep cap reached with active vertices left");
        if (glr_due(g, g->sweep)) {
            CK(glr_run(g, g->stream));
            CK(cudaMemcpyAsync(g->h_ctr, g->st.ctr, kCtrWords * 4, cudaMemcpyDeviceToHost, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            const int levels = g->h_ctr[kGlrLevels];
            active = g->h_ctr[kActiveRegions];
            g->stats.global_relabels++;
            g->stats.relabel_levels += levels;
            g->launches += 4;  // masks, the cooperative levels launch, finish, count
            if (active == 0) return MF_OK;
        } else if (br_due(g, g->sweep)) {
            mf_status bs = br_step(g, g->stream, &active, nullptr);
            if (bs != MF_OK) return bs;
            if (active == 0) return MF_OK;
        }
    }
}

mf_status mf_solve(mf_grid *g, const mf_opts *opts, mf_stats *stats) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    CK(cudaEventRecord(g->ev[0], g->stream));
    mf_status s = mf_begin(g, opts);
    if (s != MF_OK) return s;
    CK(cudaEventRecord(g->ev[1], g->stream));
    // sweep bounds: 2|B|^2+1 for ARD (Sec. 4.4), 2n^2 for PRD (Sec. 3)
    const long long nb = g->opts.kernel_variant == 2 ? (long long)g->g.n : g->boundary;
    long long cap = g->opts.max_sweeps > 0 ? g->opts.max_sweeps : std::min<long long>(2 * nb * nb + 1, 1ll << 30);
    mf_status rs = MF_OK;
    if (g->opts.graph_loop && g->begin_active != 0) rs = run_graph_loop(g, cap);
    else while (g->begin_active != 0) {  // 0: the initial labels already show a maximum preflow
        int32_t act = 0;
        rs = run_sweep(g, &act);
        if (rs != MF_OK) break;
        if (act == 0) break;
        if (g->sweep >= cap) {
            rs = fail(g, MF_ESWEEPLIMIT, "sweep cap reached with active vertices left");
            break;
        }
    }
    CK(cudaEventRecord(g->ev[2], g->stream));
    if (rs == MF_OK) {
        s = mf_finish(g);
        if (s != MF_OK) return s;
    }
    CK(cudaEventRecord(g->ev[3], g->stream));
    CK(cudaEventSynchronize(g->ev[3]));
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, g->ev[0], g->ev[1]);
    cudaEventElapsedTime(&b, g->ev[1], g->ev[2]);
    cudaEventElapsedTime(&c, g->ev[2], g->ev[3]);
    g->stats.ms_init = a;
    g->stats.ms_sweeps = b;
    g->stats.ms_cut = c;
    g->stats.ms_total = a + b + c;
    if (stats) *stats = g->stats;
    return rs;
}

// ---- batched solve --------------------------------------------------------------
// A warp per instance of a batch: st.ctr into the pinned mirror, the flow
// parts and the stage counts into the pinned record of the finished solve.
__global__ void batch_readback_kernel(const Inst *__restrict__ insts, int count) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= count) return;
    const Inst &I = insts[i];
    if (lane < kCtrWords) I.h_ctr[lane] = I.st.ctr[lane];
    mf_grid::FinishHost *f = (mf_grid::FinishHost *)I.h_fin;
    if (lane == kCtrWords) f->f0 = *I.st.flow0;
    if (lane == kCtrWords + 1) f->ft = *I.st.flow_t;
    if (lane == kCtrWords + 2) f->c = *I.c64;
}

struct BatchBufs {
    int *loop = nullptr;                   // graph loop state (kLoop* words)
    cudaStream_t cap_stream = nullptr;     // private capture stream of the graph loop
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Inst *insts = nullptr;
    int2 *regs = nullptr, *items = nullptr;
    int *type_of = nullptr, *cnt = nullptr, *head = nullptr, *sweeps = nullptr, *any = nullptr;
    unsigned char *done = nullptr;
    std::vector<cudaEvent_t> tev;          // host loop: a start / end event per kernel type
    GlrBatchBufs glr2, glr3;               // tables of the batched global relabels
    ~BatchBufs() {
        for (cudaEvent_t e : tev)
            if (e) cudaEventDestroy(e);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        void *p[] = {insts, regs, items, type_of, cnt, head, sweeps, any, done, loop};
        for (void *q : p)
            if (q) cudaFree(q);
    }
};

// The global relabel of every unfinished instance of a batch that supports it
// (or the boundary relabel where that one is due), on the batch stream (as
// after a sweep of a single solve: same sequence).  Everything is enqueued
// first; one wait then reads every relabelled instance's level count.
// Returns in *any_left the number of instances still active afterwards.
static mf_status batch_relabel(mf_grid *const *grids, int count, const Inst *insts, unsigned char *done_dev,
                               int *any_dev, int *any_left, int sweep, cudaStream_t s, double *ms_total,
                               GlrBatchBufs &glr2, GlrBatchBufs &glr3) {
    mf_grid *g = grids[0];
    std::vector<unsigned char> done(count);
    CK(cudaMemcpyAsync(done.data(), done_dev, count, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaEventRecord(g->ev[7], s));
    std::vector<int> glr;
    std::vector<GlrJob2> jobs2, jobs3;  // the global relabels of all due grids: one batched launch per dimension
    for (int i = 0; i < count; ++i) {
        mf_grid *h = grids[i];
        if (done[i]) continue;
        if (br_due(h, sweep)) {
            mf_status bs = br_step(h, s, nullptr, nullptr);
            if (bs != MF_OK) return fail(g, bs, std::string("batched boundary relabel: ") + h->err);
            continue;
        }
        if (!glr_due(h, sweep)) continue;
        GlrJob2 J{};
        J.g = h->g;
        J.st = h->st;
        J.conn = h->conn;
        J.scratch = h->cut_scratch;
        J.hout = h->h_ctr_dv + kGlrLevels;  // the level count lands in the pinned mirror
        (h->ndim == 2 ? jobs2 : jobs3).push_back(J);
        glr.push_back(i);
    }
    cudaError_t eg = glr2d_batch(jobs2, glr2, s);
    if (eg == cudaSuccess) eg = glr3d_batch(jobs3, glr3, s);
    if (eg != cudaSuccess) return fail(g, MF_ECUDA, std::string("batched global relabel: ") + cudaGetErrorString(eg));
    CK(cudaMemsetAsync(any_dev, 0, sizeof(int), s));
    batch_relabel_end_kernel<<<(count + 255) / 256, 256, 0, s>>>(insts, done_dev, any_dev, count);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(any_left, any_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(g->ev[8], s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev[7], g->ev[8]);
    *ms_total += ms;
    for (int i : glr) {
        mf_grid *h = grids[i];
        const int levels = h->h_ctr[kGlrLevels];
        h->stats.global_relabels++;
        h->stats.relabel_levels += levels;
    }
    // per dimension: masks, levels, reset, finish, count and the level counts
    if (!jobs2.empty()) g->launches += 6;
    if (!jobs3.empty()) g->launches += 6;
    return MF_OK;
}

mf_status mf_solve_batch(mf_grid *const *grids, int count, const mf_opts *opts, mf_stats *stats) {
    mf_grid *g = nullptr;  // for CK: errors are reported on the first handle
    if (!grids || count < 1) return fail(nullptr, MF_EINVAL, "grids must be a non-empty array");
    for (int i = 0; i < count; ++i)
        if (!grids[i]) return fail(nullptr, MF_EINVAL, "null grid in the batch");
    g = grids[0];
    for (int i = 0; i < count; ++i) {
        if (!grids[i]->caps_set) return fail(g, MF_ESTATE, "a grid of the batch has no capacities");
        if (grids[i]->device != g->device) return fail(g, MF_EINVAL, "all grids must be on one device");
        if (is_paper(grids[i]->conn)) return fail(g, MF_EINVAL, "the Sec. 7.1 stencils are solved one by one (mf_solve)");
        for (int j = 0; j < i; ++j)
            if (grids[j] == grids[i]) return fail(g, MF_EINVAL, "a grid appears twice in the batch");
    }
    cudaStream_t s = g->stream;
    CK(cudaEventRecord(g->ev[0], s));
    // Init of every instance on its own stream, then everything on the batch
    // stream; the cold starts on the batch stream are reset and initialised
    // by two launches for all of them
    long long cap = 0;
    std::vector<int> to_init;
    for (int i = 0; i < count; ++i) {
        // with opts.warm_start, each grid starts from its projected preflow if
        // mf_warm_start succeeded on it, and cold otherwise
        mf_opts oi;
        if (opts) oi = *opts;
        else mf_default_opts(&oi);
        if (oi.warm_start && !grids[i]->warm_ready) oi.warm_start = 0;
        bool bi = false;
        mf_status st = begin_impl(grids[i], &oi, grids[i]->stream == s, grids[i]->stream == s ? &bi : nullptr);
        if (st != MF_OK) return st;
        if (bi) to_init.push_back(i);
        if (grids[i]->stream != s) {
            cudaError_t e = cudaStreamSynchronize(grids[i]->stream);
            if (e != cudaSuccess) return fail(g, MF_ECUDA, cudaGetErrorString(e));
        }
        const long long b = grids[i]->opts.kernel_variant == 2 ? (long long)grids[i]->g.n : grids[i]->boundary;
        cap = std::max(cap, g->opts.max_sweeps > 0 ? (long long)g->opts.max_sweeps
                                                    : std::min<long long>(2 * b * b + 1, 1ll << 30));
    }
    if (!to_init.empty()) {
        std::vector<InitJob> jobs;
        std::vector<int2> units;
        for (int i : to_init) {
            mf_grid *h = grids[i];
            const int j = (int)jobs.size();
            jobs.push_back(InitJob{h->g, h->st, h->c64, h->cs, h->ct, h->nl, h->conn, (int)h->boundary});
            const long long nc = (h->g.n + kInitChunk - 1) / kInitChunk;
            for (long long c = 0; c < nc; ++c) units.push_back(make_int2(j, (int)c));
            h->launches = 2;  // its share: the reset and Init launches
        }
        InitJob *djobs = nullptr;
        int2 *dunits = nullptr;
        CK(cudaMallocAsync((void **)&djobs, jobs.size() * sizeof(InitJob), s));
        CK(cudaMallocAsync((void **)&dunits, units.size() * sizeof(int2), s));
        CK(cudaMemcpyAsync(djobs, jobs.data(), jobs.size() * sizeof(InitJob), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(dunits, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
        batch_begin_reset_kernel<<<(int)jobs.size(), 256, 0, s>>>(djobs);
        const int nu = (int)units.size();
        batch_init_kernel<<<std::min(nu, device_sms() * 16), 256, 0, s>>>(djobs, dunits, nu);
        CK(cudaGetLastError());
        CK(cudaFreeAsync(djobs, s));
        CK(cudaFreeAsync(dunits, s));
    }
    // the relabels of warm starts were left in flight: one wait for all; a grid
    // whose initial labels already show a maximum preflow makes no sweep
    CK(cudaStreamSynchronize(s));
    std::vector<unsigned char> done0(count, 0);
    for (int i = 0; i < count; ++i) {
        begin_collect(grids[i]);
        if (grids[i]->begin_active == 0) done0[i] = 1;
    }
    CK(cudaEventRecord(g->ev[1], s));
    // kernel types (connectivity, tile) and the table of all regions
    struct Type { int conn, tx, ty, tz; };
    std::vector<Type> types;
    std::vector<int> type_of(count);
    std::vector<Inst> hinst(count);
    std::vector<int2> hregs;
    for (int i = 0; i < count; ++i) {
        const mf_grid *h = grids[i];
        int t = -1;
        for (size_t k = 0; k < types.size(); ++k)
            if (types[k].conn == h->conn && types[k].tx == h->g.tx && types[k].ty == h->g.ty && types[k].tz == h->g.tz)
                t = (int)k;
        if (t < 0) {
            types.push_back({h->conn, h->g.tx, h->g.ty, h->g.tz});
            t = (int)types.size() - 1;
        }
        type_of[i] = t;
        hinst[i].g = h->g;
        hinst[i].st = h->st;
        hinst[i].c64 = h->c64;
        hinst[i].conn = h->conn;
        hinst[i].h_ctr = h->h_ctr_dv;
        hinst[i].h_fin = h->h_fin_dv;
        for (int r = 0; r < h->g.nreg; ++r) hregs.push_back(make_int2(i, r));
    }
    const int nregs = (int)hregs.size();
    const int nt = (int)types.size();
    BatchBufs B;
    CK(cudaMalloc(&B.insts, sizeof(Inst) * count));
    CK(cudaMalloc(&B.regs, sizeof(int2) * nregs));
    CK(cudaMalloc(&B.items, sizeof(int2) * (size_t)nregs * nt));
    CK(cudaMalloc(&B.type_of, sizeof(int) * count));
    CK(cudaMalloc(&B.cnt, sizeof(int) * nt));
    CK(cudaMalloc(&B.head, sizeof(int) * nt));
    CK(cudaMalloc(&B.sweeps, sizeof(int) * count));
    CK(cudaMalloc(&B.any, sizeof(int)));
    CK(cudaMalloc(&B.done, count));
    CK(cudaMemcpyAsync(B.insts, hinst.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.regs, hregs.data(), sizeof(int2) * nregs, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.type_of, type_of.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(B.sweeps, 0, sizeof(int) * count, s));
    CK(cudaMemcpyAsync(B.done, done0.data(), count, cudaMemcpyHostToDevice, s));
    const mf_opts &o = g->opts;
    SweepArgs sa{};
    sa.partial = o.partial_discharge;
    sa.max_rounds = o.max_rounds;
    sa.variant = o.kernel_variant;
    const int eb = (int)std::min<long long>(((long long)nregs + 255) / 256, device_sms() * 8);
    const int wbb = (int)std::min<long long>(((long long)nregs + 7) / 8, (long long)device_sms() * 8);
    mf_status rs = MF_OK;
    long long launches = 0;
    const int per_sweep = 6 + nt + (o.global_gap ? 1 : 0);
    // host loop: the persistent discharge launches of each kernel type are
    // timed with events (no event can be recorded inside the graph's loop body)
    std::vector<double> type_ms(nt, 0.0);
    double relabel_ms = 0.0;
    std::vector<int> type_launches(nt, 0), hcnt(nt, 0);
    if (!o.graph_loop) {
        B.tev.assign(2 * nt, nullptr);
        for (auto &e : B.tev) CK(cudaEventCreate(&e));
    }
    // one sweep of the whole batch on stream st (sweep index from the host, or
    // from sweep_dev inside a graph)
    auto enqueue_sweep = [&](cudaStream_t st, int sweep_host, const int *sweep_dev) -> cudaError_t {
        SweepArgs a = sa;
        a.sweep = sweep_host;
        a.sweep_dev = sweep_dev;
        cudaError_t e = cudaMemsetAsync(B.cnt, 0, sizeof(int) * nt, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.head, 0, sizeof(int) * nt, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(B.any, 0, sizeof(int), st);
        if (e != cudaSuccess) return e;
        batch_reset_kernel<<<(count + 255) / 256, 256, 0, st>>>(B.insts, B.done, count);
        batch_items_kernel<<<eb, 256, 0, st>>>(B.insts, B.regs, nregs, B.done, B.type_of, nregs, B.items, B.cnt);
        e = cudaGetLastError();
        for (int t = 0; t < nt && e == cudaSuccess; ++t) {
            if (!sweep_dev) e = cudaEventRecord(B.tev[2 * t], st);
            if (e == cudaSuccess)
                e = launch_discharge_batch(types[t].conn, types[t].tx, types[t].ty, types[t].tz, a.variant, B.insts,
                                           B.items + (size_t)t * nregs, B.cnt + t, B.head + t, a, device_sms() * 4,
                                           st);
            if (e == cudaSuccess && !sweep_dev) e = cudaEventRecord(B.tev[2 * t + 1], st);
        }
        if (e != cudaSuccess) return e;
        // fusion / gap / activity per connectivity of the instances (one launch per connectivity)
        for (int conn : {4, 8, 6}) {
            bool has = false;
            for (auto &ty : types) has |= ty.conn == conn;
            if (!has) continue;
            if (conn == 4) fuse_batch_kernel<4><<<wbb, 256, 0, st>>>(B.insts, B.regs, nregs, B.done);
            if (conn == 8) fuse_batch_kernel<8><<<wbb, 256, 0, st>>>(B.insts, B.regs, nregs, B.done);
            if (conn == 6) fuse_batch_kernel<6><<<wbb, 256, 0, st>>>(B.insts, B.regs, nregs, B.done);
        }
        if (o.global_gap) gap_find_batch_kernel<<<count, 1024, 0, st>>>(B.insts, B.done);
        for (int conn : {4, 8, 6}) {
            bool has = false;
            for (auto &ty : types) has |= ty.conn == conn;
            if (!has) continue;
            if (conn == 4) post_batch_kernel<4><<<wbb, 256, 0, st>>>(B.insts, B.regs, nregs, B.done);
            if (conn == 8) post_batch_kernel<8><<<wbb, 256, 0, st>>>(B.insts, B.regs, nregs, B.done);
            if (conn == 6) post_batch_kernel<6><<<wbb, 256, 0, st>>>(B.insts, B.regs, nregs, B.done);
        }
        clear_batch_kernel<<<eb, 256, 0, st>>>(B.insts, B.regs, nregs, B.done);
        batch_end_kernel<<<(count + 255) / 256, 256, 0, st>>>(B.insts, B.done, B.sweeps, B.any, count);
        return cudaGetLastError();
    };
    if (o.graph_loop) {
        // all sweeps as one CUDA graph: a while node whose body is one sweep of
        // the batch plus a loop-control kernel (continue while an instance is
        // active and the cap allows); captured on a private stream
        CK(cudaMalloc(&B.loop, sizeof(int) * kLoopWords));
        int init[kLoopWords] = {0};
        init[kLoopCap] = (int)std::min<long long>(cap, INT_MAX);
        init[kLoopPeriod] = relabel_stop_period(o, true);
        init[kLoopFirst] = std::max(0, o.global_relabel_first);
        memcpy(g->h_ctr, init, sizeof(init));
        CK(cudaMemcpyAsync(B.loop, g->h_ctr, sizeof(init), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        CK(cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking));
        CK(cudaGraphCreate(&B.graph, 0));
        cudaGraphConditionalHandle handle;
        CK(cudaGraphConditionalHandleCreate(&handle, B.graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = handle;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, B.graph, nullptr, nullptr, 0, &np));
        CK(cudaStreamBeginCaptureToGraph(B.cap_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
        cudaError_t e = enqueue_sweep(B.cap_stream, 0, &B.loop[kLoopSweep]);
        if (e == cudaSuccess) {
            batch_loop_ctl_kernel<<<1, 32, 0, B.cap_stream>>>(B.any, B.loop, handle);
            e = cudaGetLastError();
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(B.cap_stream, &captured);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return fail(g, MF_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
        CK(cudaGraphInstantiate(&B.exec, B.graph, 0));
        int loopst[kLoopWords];
        for (int before = 0;;) {
            CK(cudaGraphLaunch(B.exec, s));
            CK(cudaMemcpyAsync(g->h_ctr, B.loop, sizeof(init), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            memcpy(loopst, g->h_ctr, sizeof(loopst));
            launches += (long long)(loopst[kLoopSweep] - before) * (per_sweep + 1);
            before = loopst[kLoopSweep];
            if (!loopst[kLoopActive]) break;
            if (loopst[kLoopSweep] >= cap) {
                rs = fail(g, MF_ESWEEPLIMIT, "sweep cap reached with active vertices left in the batch");
                break;
            }
            // stopped at a multiple of the relabel period
            mf_status st = batch_relabel(grids, count, B.insts, B.done, B.any, &g->h_ctr[0], loopst[kLoopSweep], s,
                                         &relabel_ms, B.glr2, B.glr3);
            if (st != MF_OK) return st;
            if (!g->h_ctr[0]) break;
        }
    } else {
        const int P = relabel_stop_period(o, true);
        for (int sweep = 0;; ++sweep) {
            CK(enqueue_sweep(s, sweep, nullptr));
            launches += per_sweep;
            CK(cudaMemcpyAsync(g->h_ctr, B.any, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(hcnt.data(), B.cnt, sizeof(int) * nt, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int t = 0; t < nt; ++t) {
                if (!hcnt[t]) continue;  // no item of this type in the sweep
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, B.tev[2 * t], B.tev[2 * t + 1]));
                type_ms[t] += ms;
                type_launches[t]++;
            }
            if (!g->h_ctr[0]) break;
            if (sweep + 1 >= cap) {
                rs = fail(g, MF_ESWEEPLIMIT, "sweep cap reached with active vertices left in the batch");
                break;
            }
            if ((P > 0 && (sweep + 1) % P == 0) || (o.global_relabel_first > 0 && sweep + 1 == o.global_relabel_first)) {
                mf_status st = batch_relabel(grids, count, B.insts, B.done, B.any, &g->h_ctr[0], sweep + 1, s, &relabel_ms,
                                             B.glr2, B.glr3);
                if (st != MF_OK) return st;
                if (!g->h_ctr[0]) break;
            }
        }
    }
    CK(cudaEventRecord(g->ev[2], s));
    std::vector<int> hsweeps(count);
    CK(cudaMemcpyAsync(hsweeps.data(), B.sweeps, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
    // error words of every instance, then (if the loop ended normally) the cut
    // extraction of every instance, all enqueued on the batch stream with one
    // wait at the end; one launch writes every instance's counters, flow parts
    // and stage counts into its pinned records
    batch_readback_kernel<<<(count + 7) / 8, 256, 0, s>>>(B.insts, count);
    CK(cudaGetLastError());
    ++launches;
    if (rs == MF_OK) {
        // the cut closures of all grids with bit-mask cuts in one cooperative
        // launch per closure and dimension, then each grid's read-back
        std::vector<GlrJob2> j2, j3;
        std::vector<char> batched(count, 0);
        for (int i = 0; i < count; ++i) {
            mf_grid *h = grids[i];
            if (h->ndim == 3 && !glr3d_supported(h->g)) continue;
            GlrJob2 J{};
            J.g = h->g;
            J.st = h->st;
            J.conn = h->conn;
            J.scratch = h->cut_scratch;
            J.smin = h->smin;
            J.smax = h->tset;
            J.hout = h->h_fin_dv->passes;
            h->h_fin->passes[0] = h->h_fin->passes[1] = 0;
            (h->ndim == 2 ? j2 : j3).push_back(J);
            batched[i] = 1;
        }
        cudaError_t ec = cut2d_batch(j2, B.glr2, s);
        if (ec == cudaSuccess) ec = cut3d_batch(j3, B.glr3, s);
        if (ec != cudaSuccess) return fail(g, MF_ECUDA, std::string("batched cut: ") + cudaGetErrorString(ec));
        if (!j2.empty()) launches += 7;  // per closure: masks, passes, pass counts; then the bytes
        if (!j3.empty()) launches += 7;
        for (int i = 0; i < count; ++i) {
            mf_status st = finish_enqueue(grids[i], s, batched[i] != 0, false);
            if (st != MF_OK) return fail(g, st, grids[i]->err);
        }
    }
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) {
        mf_grid *h = grids[i];
        h->sweep = hsweeps[i];
        h->stats.sweeps = hsweeps[i];
        if (h->h_ctr[kError] && rs == MF_OK) rs = fail(g, MF_EROUNDLIMIT, "an Augment stage hit max_rounds");
    }
    if (rs == MF_OK)
        for (int i = 0; i < count; ++i) finish_collect(grids[i]);
    CK(cudaEventRecord(g->ev[3], s));
    CK(cudaEventSynchronize(g->ev[3]));
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, g->ev[0], g->ev[1]);
    cudaEventElapsedTime(&b, g->ev[1], g->ev[2]);
    cudaEventElapsedTime(&c, g->ev[2], g->ev[3]);
    for (int i = 0; i < count; ++i) {
        mf_grid *h = grids[i];
        h->stats.ms_init = a;
        h->stats.ms_sweeps = b;
        h->stats.ms_cut = c;
        h->stats.ms_total = a + b + c;
        if (i == 0) h->stats.launches += launches;  // launches shared by the whole batch, counted once
        h->stats.ms_discharge = type_ms[type_of[i]];
        h->stats.discharge_launches = type_launches[type_of[i]];
        h->stats.ms_relabel = relabel_ms;
        if (stats) stats[i] = h->stats;
    }
    return rs;
}

mf_status mf_region_reduction(mf_grid *g, const int32_t tile[3], uint8_t *codes, int on_device, int64_t counts[4]) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!codes) return fail(g, MF_EINVAL, "codes is NULL");
    if (is_paper(g->conn)) return fail(g, MF_EINVAL, "the region reduction is for the 4/8/6 stencils");
    if (!g->caps_set) return fail(g, MF_ESTATE, "mf_set_caps has not succeeded");
    const int saved = g->opts.max_rounds;
    g->opts.max_rounds = 0;
    bool ok = false;
    mf_status rs = reduction_run(g, tile, &ok);
    g->opts.max_rounds = saved;
    if (rs != MF_OK) return rs;
    if (!ok) return fail(g, MF_EROUNDLIMIT, "an Augment of the region reduction hit its round cap");
    CK(cudaMemcpyAsync(codes, g->red_codes, (size_t)g->g.n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (counts)
        for (int k = 0; k < 4; ++k) counts[k] = (int64_t)g->h_red[k];
    return MF_OK;
}

mf_status mf_warm_features(mf_grid *g, float *x) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!x) return fail(g, MF_EINVAL, "x is NULL");
    if (g->ndim != 2 || is_paper(g->conn)) return fail(g, MF_EINVAL, "the warm start is for 2D 4/8-connected grids");
    if (!g->caps_set) return fail(g, MF_ESTATE, "mf_set_caps has not succeeded");
    CK(launch_warm_features(g->conn, g->g, g->cs, g->ct, g->nl, x, g->stream));
    return MF_OK;
}

mf_status mf_warm_targets(mf_grid *g, float *t) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!t) return fail(g, MF_EINVAL, "t is NULL");
    if (g->ndim != 2 || is_paper(g->conn)) return fail(g, MF_EINVAL, "the warm start is for 2D 4/8-connected grids");
    if (!g->finished) return fail(g, MF_ESTATE, "no finished solve");
    CK(launch_warm_targets(g->conn, g->g, g->st, g->cs, g->ct, g->nl, t, g->stream));
    return MF_OK;
}

// The projection of a prediction, enqueued on stream st; its flag words go to
// the grid's pinned h_warm (warm_collect reads them after a wait).
static mf_status warm_enqueue(mf_grid *g, const float *pred, int32_t max_rounds, cudaStream_t st) {
    if (g->ndim != 2 || is_paper(g->conn)) return fail(g, MF_EINVAL, "the warm start is for 2D 4/8-connected grids");
    g->warm_ready = false;
    g->warm_pending = false;
    const size_t n = (size_t)g->g.n;
    if (!g->warmF) {
        CK(cudaMalloc(&g->warmF, (size_t)g->H * n * 4));
        CK(cudaMalloc(&g->warmFt, n * 4));
        CK(cudaMalloc(&g->warmE, n * 4));
        CK(cudaMallocHost((void **)&g->h_warm, 8 * 4));
    }
    if (max_rounds <= 0) max_rounds = 4096;
    CK(launch_project_init(g->conn, g->g, g->cs, g->ct, g->nl, pred, g->warmF, g->warmFt, st));
    CK(launch_project_rounds(g->conn, g->g, g->cs, g->ct, g->warmF, g->warmFt, g->warmE, &g->st.ctr[kGlrFlags],
                             max_rounds, st));
    CK(cudaMemcpyAsync(g->h_warm, &g->st.ctr[kGlrFlags], 5 * 4, cudaMemcpyDeviceToHost, st));
    g->warm_pending = true;
    return MF_OK;
}

// after the wait: the phases run (-1: no preflow; the grid then stays cold)
static int warm_collect(mf_grid *g) {
    if (!g->warm_pending) return -1;
    g->warm_pending = false;
    const int r = g->h_warm[2];
    if (r < 0) return -1;
    g->warm_rounds = r;
    g->warm_ready = true;
    return r;
}

mf_status mf_warm_start(mf_grid *g, const float *pred, int32_t max_rounds, int32_t *rounds) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!pred) return fail(g, MF_EINVAL, "pred is NULL");
    if (g->ndim != 2 || is_paper(g->conn)) return fail(g, MF_EINVAL, "the warm start is for 2D 4/8-connected grids");
    if (!g->caps_set) return fail(g, MF_ESTATE, "mf_set_caps has not succeeded");
    mf_status s = warm_enqueue(g, pred, max_rounds, g->stream);
    if (s != MF_OK) return s;
    CK(cudaStreamSynchronize(g->stream));
    const int r = warm_collect(g);
    if (r < 0) {
        if (rounds) *rounds = max_rounds <= 0 ? 4096 : max_rounds;
        return fail(g, MF_EROUNDLIMIT, "projection did not reach a preflow within max_rounds");
    }
    if (rounds) *rounds = r;
    return MF_OK;
}

mf_status mf_warm_start_batch(mf_grid *const *grids, int count, const float *const *preds, int32_t max_rounds,
                              int32_t *rounds) {
    if (!grids || !preds || count < 1) return fail(nullptr, MF_EINVAL, "grids and preds must be non-empty arrays");
    mf_grid *g = grids[0];
    if (!g) return fail(nullptr, MF_EINVAL, "null grid in the batch");
    cudaStream_t s = g->stream;
    for (int i = 0; i < count; ++i) {
        mf_grid *h = grids[i];
        if (!h) return fail(g, MF_EINVAL, "null grid in the batch");
        if (!preds[i]) continue;
        if (h->ndim != 2) return fail(g, MF_EINVAL, "the warm start is for 2D grids");
        if (!h->caps_set) return fail(g, MF_ESTATE, "a grid of the batch has no capacities");
        if (h->device != g->device) return fail(g, MF_EINVAL, "all grids must be on one device");
        if (h->stream != s) CK(cudaStreamSynchronize(h->stream));  // its earlier work precedes the batch stream's
        mf_status st = warm_enqueue(h, preds[i], max_rounds, s);
        if (st != MF_OK) return fail(g, st, h->err);
    }
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) {
        const int r = preds[i] ? warm_collect(grids[i]) : -1;
        if (rounds) rounds[i] = r;
    }
    return MF_OK;
}

mf_status mf_get_cut(mf_grid *g, uint8_t *out, int which, int on_device) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!out || (which != 0 && which != 1)) return fail(g, MF_EINVAL, "bad output or which");
    if (!g->finished) return fail(g, MF_ESTATE, "no finished solve");
    CK(cudaMemcpyAsync(out, which == 0 ? g->smin : g->tset, (size_t)g->g.n,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    if (!on_device) CK(cudaStreamSynchronize(g->stream));
    return MF_OK;
}

mf_status mf_get_cuts_batch(mf_grid *const *grids, int count, int which, uint8_t *const *out, int on_device,
                            int64_t *flows) {
    if (!grids || count < 1 || !out || (which != 0 && which != 1)) return fail(nullptr, MF_EINVAL, "bad batch arguments");
    for (int i = 0; i < count; ++i)
        if (!grids[i] || !out[i]) return fail(nullptr, MF_EINVAL, "null grid or output in the batch");
    mf_grid *g = grids[0];
    for (int i = 0; i < count; ++i) {
        mf_grid *h = grids[i];
        if (!h->finished) return fail(g, MF_ESTATE, std::string("grid ") + std::to_string(i) + " has no finished solve");
        CK(cudaMemcpyAsync(out[i], which == 0 ? h->smin : h->tset, (size_t)h->g.n,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
        if (flows) flows[i] = h->stats.flow_value;
    }
    if (!on_device) CK(sync_streams(grids, count));
    return MF_OK;
}

mf_status mf_flow_value(mf_grid *g, int64_t *out) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!out) return fail(g, MF_EINVAL, "out is NULL");
    if (!g->begun) return fail(g, MF_ESTATE, "no solve");
    if (g->flow_cached) {  // read back with the finished solve's results
        *out = g->stats.flow_value;
        return MF_OK;
    }
    long long f0 = 0;
    unsigned long long ft = 0;
    CK(cudaMemcpyAsync(&f0, g->st.flow0, 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(&ft, g->st.flow_t, 8, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    *out = f0 + (long long)ft;
    return MF_OK;
}

mf_status mf_certify(mf_grid *g, int64_t *cut_capacity, int64_t *violations, int32_t *certified) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!g->finished) return fail(g, MF_ESTATE, "no finished solve");
    // three 64-bit sums in the last six counter words (unused once a solve has finished)
    unsigned long long *sums = (unsigned long long *)&g->st.ctr[kCtrWords - 6];
    CK(cudaMemsetAsync(sums, 0, 3 * 8, g->stream));
    CK(DISPATCH(g->conn, launch_certify, g, sums));
    unsigned long long h[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    int64_t flow = 0;
    mf_status s = mf_flow_value(g, &flow);
    if (s != MF_OK) return s;
    // the constant of the reduction: cut edges between the merged vertex sets
    const int64_t k = g->reduced ? (int64_t)g->red_konst : 0;
    if (cut_capacity) *cut_capacity = (int64_t)h[0] + k;
    if (violations) *violations = (int64_t)h[2];
    if (certified) *certified = h[2] == 0 && (int64_t)h[0] + k == flow && (int64_t)h[1] + k == flow;
    return MF_OK;
}

mf_status mf_get_residual(mf_grid *g, int32_t *res, int32_t *tres, int32_t *exc, int on_device) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!g->begun) return fail(g, MF_ESTATE, "no solve");
    const size_t n = (size_t)g->g.n;
    (void)on_device;  // unified addressing: the direction follows from the pointers (planes may be host memory)
    const cudaMemcpyKind k = cudaMemcpyDefault;
    if (res) CK(cudaMemcpyAsync(res, g->st.cap, (size_t)g->N * n * 4, k, g->stream));
    if (tres) CK(cudaMemcpyAsync(tres, g->st.tcap, n * 4, k, g->stream));
    if (exc) CK(cudaMemcpyAsync(exc, g->st.exc, n * 4, k, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return MF_OK;
}

mf_status mf_get_flow(mf_grid *g, int32_t *residual_out) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (!residual_out) return MF_OK;
    return mf_get_residual(g, residual_out, nullptr, nullptr, 0);
}

mf_status mf_get_labels(mf_grid *g, int32_t *lab, int32_t *d_inf, int on_device) {
    if (!g) return fail(nullptr, MF_EINVAL, "grid is NULL");
    if (d_inf) *d_inf = g->g.dinf;
    (void)on_device;  // cudaMemcpyDefault tells host from device buffers itself
    if (lab) {
        if (!g->begun) return fail(g, MF_ESTATE, "no solve");
        CK(cudaMemcpyAsync(lab, g->st.lab, (size_t)g->g.n * 4, cudaMemcpyDefault, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    }
    return MF_OK;
}

}  // extern "C"
