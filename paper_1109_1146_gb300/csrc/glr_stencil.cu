// Exact region-distance relabel (the global relabel heuristic) for the grids
// with the longer displacements of the Sec. 7.1 synthetic networks, where the
// bit-mask relabels (unit shifts) do not apply.
//
// d*(u) = the least number of inter-region arcs on a residual path from u to
// t (the region distance of Sec. 4.1, eq. 3).  Level sets S_0 ⊆ S_1 ⊆ ...:
// S_0 = vertices that reach t through residual arcs inside their own region;
// S_l adds every vertex with a residual inter-region arc into S_{l-1}, then
// closes each region under its inner residual arcs.  A vertex first reached
// at level l gets d := max(d, l); vertices never reached get d_inf (as the 2D
// and 3D relabels).  One thread block per region and level, the region's set
// in shared memory (one byte per vertex of the tile); all levels in one
// cooperative launch with a grid barrier per level.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "mf_internal.cuh"

namespace mf {

namespace cg = cooperative_groups;

// level `level` of region r: S_l(r) from S_{l-1} (in; unused at level 0) into
// out; raises the labels of the vertices it adds; returns whether it added any
template <int CONN, int TX, int TY>
__device__ bool stencil_region_level(const Geom &g, const DevState &st, int r, const unsigned char *in,
                                     unsigned char *out, int level, unsigned char *m) {
    constexpr int N = arcs_of(CONN), V = TX * TY;
    constexpr int SX = TX == 64 ? 6 : 5;  // log2 TX
    const int rx = r % g.RX, ry = r / g.RX;
    const size_t n = (size_t)g.n;
    for (int i = threadIdx.x; i < V; i += blockDim.x) {
        const int x = rx * TX + (i & (TX - 1)), y = ry * TY + (i >> SX);
        unsigned char s = 0;
        if (x < g.X && y < g.Y) {
            const size_t v = (size_t)y * g.X + x;
            if (level == 0) {
                s = st.tcap[v] > 0;
            } else {
                s = in[v];
#pragma unroll
                for (int d = 0; d < N && !s; ++d) {  // a residual arc into S_{l-1} of another region
                    const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d);
                    if (wx < 0 || wx >= g.X || wy < 0 || wy >= g.Y) continue;
                    if (wx / TX == rx && wy / TY == ry) continue;
                    s = in[(size_t)wy * g.X + wx] && st.cap[(size_t)d * n + v] > 0;
                }
            }
        }
        m[i] = s;
    }
    __syncthreads();
    // closure inside the region (monotone: a stale read only delays)
    for (;;) {
        int ch = 0;
        for (int i = threadIdx.x; i < V; i += blockDim.x) {
            if (m[i]) continue;
            const int lx = i & (TX - 1), ly = i >> SX;
            const int x = rx * TX + lx, y = ry * TY + ly;
            if (x >= g.X || y >= g.Y) continue;
            const size_t v = (size_t)y * g.X + x;
#pragma unroll
            for (int d = 0; d < N; ++d) {
                const int nx = lx + arc_dx(CONN, d), ny = ly + arc_dy(CONN, d);
                if (nx < 0 || nx >= TX || ny < 0 || ny >= TY) continue;
                if (x + arc_dx(CONN, d) >= g.X || y + arc_dy(CONN, d) >= g.Y) continue;
                if (m[ny * TX + nx] && st.cap[(size_t)d * n + v] > 0) {
                    m[i] = 1;
                    ch = 1;
                    break;
                }
            }
        }
        if (!__syncthreads_or(ch)) break;
    }
    int grew = 0;
    for (int i = threadIdx.x; i < V; i += blockDim.x) {
        const int x = rx * TX + (i & (TX - 1)), y = ry * TY + (i >> SX);
        if (x >= g.X || y >= g.Y) continue;
        const size_t v = (size_t)y * g.X + x;
        out[v] = m[i];
        if (level > 0 && m[i] && !in[v]) {
            grew = 1;
            if (st.lab[v] < level) st.lab[v] = level;
        }
    }
    return __syncthreads_or(grew) != 0;
}

// all levels in one cooperative launch; flags[3] triple-buffered "grew" words
template <int CONN, int TX, int TY>
__global__ void stencil_glr_levels_kernel(const Geom g, const DevState st, unsigned char *A, unsigned char *B,
                                          int *flags, int *levels_out, int max_levels) {
    cg::grid_group grid = cg::this_grid();
    __shared__ unsigned char m[TX * TY];
    for (int r = blockIdx.x; r < g.nreg; r += gridDim.x) stencil_region_level<CONN, TX, TY>(g, st, r, nullptr, B, 0, m);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flags[1] = 0;
        flags[2] = 0;
    }
    grid.sync();
    int level = 1;
    for (; level < max_levels; ++level) {
        const unsigned char *in = (level & 1) ? B : A;
        unsigned char *out = (level & 1) ? A : B;
        bool grew = false;
        for (int r = blockIdx.x; r < g.nreg; r += gridDim.x)
            grew |= stencil_region_level<CONN, TX, TY>(g, st, r, in, out, level, m);
        if (grew && threadIdx.x == 0) atomicOr(&flags[level % 3], 1);
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(level + 1) % 3] = 0;
        grid.sync();
        if (!*(volatile int *)&flags[level % 3]) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *levels_out = level + 1;
}

// unreached vertices get d_inf; boundary-label histogram and region activity
template <int CONN>
__global__ void stencil_glr_finish_kernel(const Geom g, const DevState st, const unsigned char *A,
                                          const unsigned char *B) {
    constexpr int SB = 2048;
    const int last = st.ctr[kGlrLevels] - 1;  // level 0 and the even levels wrote B
    const unsigned char *S = (last % 2 == 1) ? A : B;
    __shared__ int sh[SB];
    for (int b = threadIdx.x; b < SB; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < (size_t)g.n; v += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(v / g.X), x = (int)(v - (size_t)y * g.X);
        int l = st.lab[v];
        if (!S[v]) {
            l = g.dinf;
            st.lab[v] = l;
        }
        if (l >= g.dinf) continue;
        const int r = (y >> g.sy) * g.RX + (x >> g.sx);
        if (st.exc[v] > 0) st.active[r] = 1;
        bool inB = false;
#pragma unroll
        for (int d = 0; d < arcs_of(CONN); ++d) {
            const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d);
            if (wx < 0 || wx >= g.X || wy < 0 || wy >= g.Y) continue;
            inB |= (wy >> g.sy) * g.RX + (wx >> g.sx) != r;
        }
        if (!inB) continue;
        if (l < SB) atomicAdd(&sh[l], 1);
        else atomicAdd(&st.hist[l < kHistBins ? l : kHistBins], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < SB; b += blockDim.x)
        if (sh[b]) atomicAdd(&st.hist[b], sh[b]);
}

__global__ void stencil_glr_count_kernel(const DevState st, int nreg) {
    int c = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) c += st.active[r] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st.ctr[kActiveRegions], c);
}

template <int CONN, int TX, int TY>
static cudaError_t stencil_glr_impl(const Geom &g, const DevState &st, void *scratch, cudaStream_t s) {
    unsigned char *A = (unsigned char *)scratch, *B = A + g.n;
    int max_blocks = 0;
    {
        const cudaError_t e_mb = coop_max_blocks((const void *)stencil_glr_levels_kernel<CONN, TX, TY>, 256, 0, &max_blocks);
        if (e_mb != cudaSuccess) return e_mb;
    }
    const int nblocks = std::max(1, std::min(g.nreg, max_blocks));
    int *flags = &st.ctr[kGlrFlags];
    int *lvl = &st.ctr[kGlrLevels];
    int max_levels = 1 << 20;
    Geom gg = g;
    DevState ss = st;
    void *args[] = {&gg, &ss, &A, &B, &flags, &lvl, &max_levels};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)stencil_glr_levels_kernel<CONN, TX, TY>, dim3(nblocks),
                                                dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(st.hist, 0, (kHistBins + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.active, 0, (size_t)g.nreg, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st.ctr[kActiveRegions], 0, 4, s);
    if (e != cudaSuccess) return e;
    const int nb = (int)std::min<size_t>(((size_t)g.n + 255) / 256, device_sms() * 32);
    stencil_glr_finish_kernel<CONN><<<nb, 256, 0, s>>>(g, st, A, B);
    stencil_glr_count_kernel<<<(g.nreg + 255) / 256, 256, 0, s>>>(st, g.nreg);
    return cudaGetLastError();
}

bool stencil_glr_supported(int conn, const Geom &g) {
    return is_paper(conn) && g.tz == 1 &&
           ((g.tx == 32 && g.ty == 32) || (conn == 108 && g.tx == 64 && (g.ty == 32 || g.ty == 64)));
}

size_t stencil_glr_scratch_bytes(const Geom &g) { return 2 * (size_t)g.n; }

cudaError_t stencil_glr(int conn, const Geom &g, const DevState &st, void *scratch, cudaStream_t s) {
    if (g.tx == 64) {  // connectivity 8 only
        if (conn != 108) return cudaErrorInvalidValue;
        return g.ty == 64 ? stencil_glr_impl<108, 64, 64>(g, st, scratch, s) : stencil_glr_impl<108, 64, 32>(g, st, scratch, s);
    }
    switch (conn) {
        case 108: return stencil_glr_impl<108, 32, 32>(g, st, scratch, s);
        case 112: return stencil_glr_impl<112, 32, 32>(g, st, scratch, s);
        case 116: return stencil_glr_impl<116, 32, 32>(g, st, scratch, s);
        case 120: return stencil_glr_impl<120, 32, 32>(g, st, scratch, s);
        case 124: return stencil_glr_impl<124, 32, 32>(g, st, scratch, s);
        case 128: return stencil_glr_impl<128, 32, 32>(g, st, scratch, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mf
