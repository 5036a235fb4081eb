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
//   capacities stay respected; a vertex that cannot be fixed, or a phase cap,
//   ends with a cold start instead.  The rounds are computed tile by tile
//   (see project_tiles_kernel), which reaches the same preflow.
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

// The trims, organised by tiles.  Let D_v be the total outflow a vertex has
// trimmed; the greedy order (sink flow first, then arcs 0..N-1) makes its
// outflows a function of D_v alone, and its excess grows with D_v and falls
// as its neighbours trim (their outflows are its inflows).  A synchronous
// round sets D_v := max(D_v, T_v(D)), T_v(D) = the trim that would make its
// excess 0 given its neighbours' trims, a map that is monotone in D.  From
// D = 0 such updates can only climb to the least fixed point of
// D = max(0, T(D)), and they stop exactly there, in whatever order they are
// applied (stale neighbour values only give smaller steps).  So the rounds
// below, local to 32x32 tiles, reach bit for bit the preflow the synchronous
// rounds reach.  A tile iterates its vertices in shared memory until none of
// them has a deficit, given the flows on the edges into it from outside;
// phases of all tiles repeat (one grid barrier each) until no tile changed
// an edge whose other end lies in another tile.  A vertex whose deficit
// exceeds all its remaining outflow can never be fixed (its trims are at
// their maximum and its inflows can only fall): the projection fails.
// Only the tail of an edge (the endpoint its flow leaves) ever lowers it, so
// every flow value has one writer.
constexpr int kProjTile = 32;

template <int CONN>
__global__ void __launch_bounds__(256) project_tiles_kernel(const Geom g, const int *cs, const int *ct, int *F, int *ft,
                                                            int *E, int *flags, int max_phases) {
    constexpr int H = CONN / 2, TP = kProjTile, EW = TP + 2, EXT = EW * EW;
    cg::grid_group grid = cg::this_grid();
    __shared__ int Fs[H][EXT];   // flows of the edges whose lower endpoint is in the tile or its ring
    __shared__ int F0[H][EXT];   // as loaded (only changed values are written back)
    __shared__ int fts[TP * TP];
    __shared__ int bs[TP * TP];  // cs - min(cs, ct)
    const size_t n = (size_t)g.n;
    const int tid = threadIdx.x;
    const int TXn = (g.X + TP - 1) / TP, TYn = (g.Y + TP - 1) / TP, ntiles = TXn * TYn;
    int phase = 0;
    for (;; ++phase) {
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int ox = (t % TXn) * TP, oy = (t / TXn) * TP;
            for (int c = tid; c < EXT; c += blockDim.x) {
                const int x = ox - 1 + c % EW, y = oy - 1 + c / EW;
                const bool in = ingrid2(g, x, y);
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const int f = in ? F[h * n + (size_t)y * g.X + x] : 0;
                    Fs[h][c] = f;
                    F0[h][c] = f;
                }
            }
            for (int i = tid; i < TP * TP; i += blockDim.x) {
                const int x = ox + i % TP, y = oy + i / TP;
                const bool in = ingrid2(g, x, y);
                const size_t v = (size_t)y * g.X + x;
                fts[i] = in ? ft[v] : 0;
                bs[i] = in ? cs[v] - min(cs[v], ct[v]) : 0;
            }
            __syncthreads();
            int cross = 0, bad = 0, trimmed = 0;
            for (int it = 0;; ++it) {
                int changed = 0;
                for (int i = tid; i < TP * TP; i += blockDim.x) {
                    const int lx = i % TP, ly = i / TP;
                    if (!ingrid2(g, ox + lx, oy + ly)) continue;
                    const int c = (ly + 1) * EW + (lx + 1);
                    long long e = (long long)bs[i] - fts[i];
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        e -= Fs[h][c];
                        e += Fs[h][c - fwd_dx(CONN, h) - fwd_dy(CONN, h) * EW];
                    }
                    if (e >= 0) continue;
                    int def = (int)-e;
                    changed = 1;
                    int r = min(fts[i], def);
                    fts[i] -= r;
                    def -= r;
#pragma unroll
                    for (int d = 0; d < CONN; ++d) {
                        if (def == 0) break;
                        const int h = d >> 1;
                        // the edge of arc d: stored at c (d even) or at its tail cell (d odd)
                        const int cc = (d & 1) ? c - fwd_dx(CONN, h) - fwd_dy(CONN, h) * EW : c;
                        const int f = Fs[h][cc];
                        const int out = (d & 1) ? -f : f;  // v's outflow on this edge
                        if (out <= 0) continue;
                        r = min(out, def);
                        Fs[h][cc] = (d & 1) ? f + r : f - r;
                        def -= r;
                        const int nx = lx + arc_dx(CONN, d), ny = ly + arc_dy(CONN, d);
                        if (nx < 0 || nx >= TP || ny < 0 || ny >= TP) cross = 1;  // the head is in another tile
                    }
                    if (def > 0) bad = 1;
                }
                if (!__syncthreads_or(changed)) break;
                trimmed = 1;
                if (it >= (1 << 16)) {  // never expected: report a failure, not a false convergence
                    bad = 1;
                    break;
                }
            }
            bad = __syncthreads_or(bad);
            cross = __syncthreads_or(cross);
            // write back what this tile's vertices trimmed (they are the tails)
            for (int c = tid; c < EXT; c += blockDim.x) {
                const int x = ox - 1 + c % EW, y = oy - 1 + c / EW;
                if (!ingrid2(g, x, y)) continue;
#pragma unroll
                for (int h = 0; h < H; ++h)
                    if (Fs[h][c] != F0[h][c]) F[h * n + (size_t)y * g.X + x] = Fs[h][c];
            }
            for (int i = tid; i < TP * TP; i += blockDim.x) {
                const int x = ox + i % TP, y = oy + i / TP;
                if (ingrid2(g, x, y)) ft[(size_t)y * g.X + x] = fts[i];
            }
            if (tid == 0) {
                if (cross) atomicOr(&flags[phase & 1], 1);
                if (bad) atomicOr(&flags[3], 1);
                if (trimmed) atomicOr(&flags[4], 1);
            }
            __syncthreads();  // the shared arrays are reused by the next tile
        }
        grid.sync();
        const int cross = *(volatile int *)&flags[phase & 1];
        const int bad = *(volatile int *)&flags[3];
        if (bad || !cross || phase + 1 >= max_phases) {
            // phases that trimmed (0: the prediction already was a preflow)
            const int any = *(volatile int *)&flags[4];
            if (blockIdx.x == 0 && tid == 0) flags[2] = (bad || cross) ? -1 : (any ? phase + 1 : 0);
            break;
        }
        if (blockIdx.x == 0 && tid == 0) flags[(phase + 1) & 1] = 0;
        grid.sync();  // the cleared word is seen before the next phase sets it
    }
    grid.sync();
    // excess of the final preflow
    for (size_t v = blockIdx.x * (size_t)blockDim.x + tid; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const int px = (int)(v % g.X), py = (int)(v / g.X);
        long long e = (long long)cs[v] - min(cs[v], ct[v]) - ft[v];
#pragma unroll
        for (int h = 0; h < CONN / 2; ++h) {
            e -= F[h * n + v];
            const int wx = px - fwd_dx(CONN, h), wy = py - fwd_dy(CONN, h);
            if (ingrid2(g, wx, wy)) e += F[h * n + (size_t)wy * g.X + wx];
        }
        E[v] = (int)e;
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
    const size_t b = ((size_t)g.n + 255) / 256, cap = (size_t)device_sms() * 16;
    return (int)(b < cap ? (b ? b : 1) : cap);
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
    const void *kern = conn == 4 ? (const void *)project_tiles_kernel<4>
                     : conn == 8 ? (const void *)project_tiles_kernel<8> : nullptr;
    if (!kern) return cudaErrorInvalidValue;
    int max_blocks = 0;
    cudaError_t e = coop_max_blocks(kern, 256, 0, &max_blocks);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((g.X + kProjTile - 1) / kProjTile) * ((g.Y + kProjTile - 1) / kProjTile);
    const int blocks = (int)std::max<long long>(1, std::min<long long>(tiles, max_blocks));
    e = cudaMemsetAsync(flags, 0, 5 * sizeof(int), s);
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
