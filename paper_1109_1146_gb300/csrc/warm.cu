// Learned warm start: network inputs and training targets from a grid, and
// the projection of predicted flows to a valid preflow that replaces the
// zero flow of Init (Sec. 2) before the sweeps start.
//
// Channels (connectivity N = 4 or 8, scale S = kWarmScale):
//   features x[2+N][n]: cs/S, ct/S, then the capacity of the edge carried by
//                       arc d at v, for d = 0..N-1, divided by S;
//   targets  t[N+2][n]: flow out of v along arc d (d = 0..N-1), the flow taken
//                       from s and the flow sent into t, all / S; the s and t
//                       flows are those of the reduced network, i.e. without
//                       the min(cs, ct) that Init routes straight through v.
// Projection of a prediction p (same layout as the targets):
//   edge flow f(v, v+h-th offset) = round(S p[2h][v]) clamped to [-c, c];
//   sink flow ft(v) = round(S p[N+1][v]) clamped to [0, ct - min(cs, ct)];
//   every s-link saturated (the s-flow prediction is not used: ARD never pushes
//   back to s, so an unsaturated s-link could not be completed later);
//   then, in synchronous rounds, every vertex with negative excess lowers its
//   own outflow (sink flow first, then arcs 0..N-1) by its deficit, until no
//   excess is negative.  Lowering an outflow only moves flow toward zero, so
//   capacities stay respected; a round cap ends with a cold start instead.
#include <algorithm>
#include <cstdint>

#include <cooperative_groups.h>

#include "mf_internal.cuh"

namespace cg = cooperative_groups;

namespace mf {

constexpr float kWarmScale = 100.f;

__device__ __forceinline__ bool ingrid2(const Geom &g, int x, int y) { return x >= 0 && x < g.X && y >= 0 && y < g.Y; }

// capacity of the edge carried by arc d at (x,y), 0 outside the grid
template <int CONN>
__device__ __forceinline__ int edge_cap(const Geom &g, const int *nl, int x, int y, int d) {
    const int h = d >> 1;
    const size_t n = (size_t)g.n;
    const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d);
    if (!ingrid2(g, wx, wy)) return 0;
    return (d & 1) ? nl[h * n + (size_t)wy * g.X + wx] : nl[h * n + (size_t)y * g.X + x];
}

template <int CONN>
__global__ void warm_features_kernel(const Geom g, const int *cs, const int *ct, const int *nl, float *x) {
    const size_t n = (size_t)g.n;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const int px = (int)(v % g.X), py = (int)(v / g.X);
        x[v] = cs[v] / kWarmScale;
        x[n + v] = ct[v] / kWarmScale;
#pragma unroll
        for (int d = 0; d < CONN; ++d) x[(2 + d) * n + v] = edge_cap<CONN>(g, nl, px, py, d) / kWarmScale;
    }
}

template <int CONN>
__global__ void warm_targets_kernel(const Geom g, const DevState st, const int *cs, const int *ct, const int *nl,
                                    float *t) {
    const size_t n = (size_t)g.n;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const int px = (int)(v % g.X), py = (int)(v / g.X);
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const int c = edge_cap<CONN>(g, nl, px, py, d);
            t[d * n + v] = (c - st.cap[d * n + v]) / kWarmScale;  // f(v, v+D(d)) = c - residual
        }
        const int m = min(cs[v], ct[v]);
        t[CONN * n + v] = (cs[v] - m - st.exc[v]) / kWarmScale;
        t[(CONN + 1) * n + v] = (ct[v] - m - st.tcap[v]) / kWarmScale;
    }
}

// initial edge flows F[h][v] and sink flows ft[v] from a prediction
template <int CONN>
__global__ void project_init_kernel(const Geom g, const int *cs, const int *ct, const int *nl, const float *p, int *F,
                                    int *ft) {
    const size_t n = (size_t)g.n;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const int px = (int)(v % g.X), py = (int)(v / g.X);
#pragma unroll
        for (int h = 0; h < CONN / 2; ++h) {
            const int c = edge_cap<CONN>(g, nl, px, py, 2 * h);
            float f = rintf(p[(2 * h) * n + v] * kWarmScale);
            f = fminf(fmaxf(f, (float)-c), (float)c);
            F[h * n + v] = c ? (int)f : 0;
        }
        const int ctr = ct[v] - min(cs[v], ct[v]);
        float q = rintf(p[(CONN + 1) * n + v] * kWarmScale);
        q = fminf(fmaxf(q, 0.f), (float)ctr);
        ft[v] = (int)q;
    }
}

// a vertex with a deficit lowers its own outflows (an edge carries flow one
// way, so only its tail ever lowers it: no two threads write one edge)
template <int CONN>
__device__ __forceinline__ void trim_vertex(const Geom &g, size_t v, const int *E, int *F, int *ft) {
    const size_t n = (size_t)g.n;
    int def = -E[v];
    if (def <= 0) return;
    const int px = (int)(v % g.X), py = (int)(v / g.X);
    int r = min(ft[v], def);
    ft[v] -= r;
    def -= r;
#pragma unroll
    for (int d = 0; d < CONN; ++d) {
        if (def == 0) break;
        const int h = d >> 1;
        if (!(d & 1)) {
            const int f = F[h * n + v];
            if (f > 0) {
                r = min(f, def);
                F[h * n + v] = f - r;
                def -= r;
            }
        } else {
            const int wx = px - fwd_dx(CONN, h), wy = py - fwd_dy(CONN, h);
            if (!ingrid2(g, wx, wy)) continue;
            const size_t w = (size_t)wy * g.X + wx;
            const int f = F[h * n + w];  // flow w -> v; negative means v -> w
            if (f < 0) {
                r = min(-f, def);
                F[h * n + w] = f + r;
                def -= r;
            }
        }
    }
}

// All projection rounds in one cooperative launch: each round computes every
// excess (flagging a negative one), and if some excess is negative and rounds
// remain, trims.  flags[0..1] alternate between rounds (the host zeroes both
// first); flags[2] receives the number of trim rounds made, or -1 if
// max_rounds trims left a negative excess.  Every loop is bounded by
// max_rounds; the grid is co-resident, so every grid.sync returns.
template <int CONN>
__global__ void project_rounds_kernel(const Geom g, const int *cs, const int *ct, int *F, int *ft, int *E, int *flags,
                                      int max_rounds) {
    cg::grid_group grid = cg::this_grid();
    const size_t n = (size_t)g.n;
    for (int r = 0;; ++r) {
        int any = 0;
        for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
            const int px = (int)(v % g.X), py = (int)(v / g.X);
            long long e = (long long)cs[v] - min(cs[v], ct[v]) - ft[v];
#pragma unroll
            for (int h = 0; h < CONN / 2; ++h) {
                e -= F[h * n + v];
                const int wx = px - fwd_dx(CONN, h), wy = py - fwd_dy(CONN, h);
                if (ingrid2(g, wx, wy)) e += F[h * n + (size_t)wy * g.X + wx];
            }
            E[v] = (int)e;
            any |= e < 0;
        }
        if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(&flags[r & 1], 1);
        grid.sync();
        const int neg = *(volatile int *)&flags[r & 1];
        if (!neg || r >= max_rounds) {
            if (blockIdx.x == 0 && threadIdx.x == 0) flags[2] = neg ? -1 : r;
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(r + 1) & 1] = 0;  // read by nobody since the last sync
        for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
            trim_vertex<CONN>(g, v, E, F, ft);
        grid.sync();
    }
}

// Init from the projected preflow: residuals, sink residuals, excess, labels 0,
// active regions, flow0 = sum min(cs, ct) and the initial flow into t
template <int CONN>
__global__ void warm_init_kernel(const Geom g, const DevState st, const int *cs, const int *ct, const int *nl,
                                 const int *F, const int *ft, const int *E) {
    const size_t n = (size_t)g.n;
    long long part0 = 0, partt = 0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const int px = (int)(v % g.X), py = (int)(v / g.X);
        const int m = min(cs[v], ct[v]);
        part0 += m;
        partt += ft[v];
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const int c = edge_cap<CONN>(g, nl, px, py, d);
            int r = 0;
            if (c) {
                const int h = d >> 1;
                if (!(d & 1)) {
                    r = c - F[h * n + v];
                } else {
                    const int wx = px - fwd_dx(CONN, h), wy = py - fwd_dy(CONN, h);
                    r = c + F[h * n + (size_t)wy * g.X + wx];
                }
            }
            st.cap[d * n + v] = r;
        }
        st.tcap[v] = ct[v] - m - ft[v];
        st.exc[v] = E[v];
        st.lab[v] = 0;
        if (E[v] > 0) st.active[((py >> g.sy) * g.RX) + (px >> g.sx)] = 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        part0 += __shfl_down_sync(0xffffffffu, part0, o);
        partt += __shfl_down_sync(0xffffffffu, partt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (part0) atomicAdd((unsigned long long *)st.flow0, (unsigned long long)part0);
        if (partt) atomicAdd(st.flow_t, (unsigned long long)partt);
    }
}

static int nblk(const Geom &g) {
    const size_t b = ((size_t)g.n + 255) / 256;
    return (int)(b < device_sms() * 16 ? (b ? b : 1) : device_sms() * 16);
}

#define WARM_DISPATCH(conn, kern, ...)                                            \
    do {                                                                          \
        if ((conn) == 4) kern<4><<<nblk(g), 256, 0, s>>>(__VA_ARGS__);            \
        else if ((conn) == 8) kern<8><<<nblk(g), 256, 0, s>>>(__VA_ARGS__);       \
        else return cudaErrorInvalidValue;                                        \
        return cudaGetLastError();                                                \
    } while (0)

cudaError_t launch_warm_features(int conn, const Geom &g, const int *cs, const int *ct, const int *nl, float *x,
                                 cudaStream_t s) {
    WARM_DISPATCH(conn, warm_features_kernel, g, cs, ct, nl, x);
}
cudaError_t launch_warm_targets(int conn, const Geom &g, const DevState &st, const int *cs, const int *ct,
                                const int *nl, float *t, cudaStream_t s) {
    WARM_DISPATCH(conn, warm_targets_kernel, g, st, cs, ct, nl, t);
}
cudaError_t launch_project_init(int conn, const Geom &g, const int *cs, const int *ct, const int *nl, const float *p,
                                int *F, int *ft, cudaStream_t s) {
    WARM_DISPATCH(conn, project_init_kernel, g, cs, ct, nl, p, F, ft);
}
cudaError_t launch_project_rounds(int conn, const Geom &g, const int *cs, const int *ct, int *F, int *ft, int *E,
                                  int *flags, int max_rounds, cudaStream_t s) {
    const void *kern = conn == 4 ? (const void *)project_rounds_kernel<4>
                     : conn == 8 ? (const void *)project_rounds_kernel<8> : nullptr;
    if (!kern) return cudaErrorInvalidValue;
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    const size_t want = ((size_t)g.n + 255) / 256;
    const int blocks = (int)std::min<size_t>(want ? want : 1, (size_t)per_sm * sms);
    e = cudaMemsetAsync(flags, 0, 3 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    Geom gg = g;
    const int *a_cs = cs, *a_ct = ct;
    int mr = max_rounds;
    void *args[] = {&gg, (void *)&a_cs, (void *)&a_ct, &F, &ft, &E, &flags, &mr};
    return cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(256), args, 0, s);
}
cudaError_t launch_warm_init(int conn, const Geom &g, const DevState &st, const int *cs, const int *ct, const int *nl,
                             const int *F, const int *ft, const int *E, cudaStream_t s) {
    WARM_DISPATCH(conn, warm_init_kernel, g, st, cs, ct, nl, F, ft, E);
}

}  // namespace mf
