// Exact region-distance relabel (the global relabel heuristic) and the cut
// closures for 3D 6-connected grids tiled by 32-voxel-wide regions (32x16x8,
// 32x8x8, 32x8x4, 32x4x4, 32x8x2).
//
// d*(u) = the least number of inter-region arcs on a residual path from u to
// t (the region distance of Sec. 4.1, eq. 3).  Level sets S_0 ⊆ S_1 ⊆ ...:
// S_0 = vertices that reach t through arcs inside their own region; S_l adds
// every vertex with a residual inter-region arc into S_{l-1}, then closes each
// region under its inner arcs.  A vertex first reached at level l gets
// d := max(d, l); vertices never reached get d_inf.  Raising labels to a
// valid lower bound of the distance keeps the labeling valid and monotone
// (the argument of Sec. 6.1).
//
// Layout: one 32-bit word per x-run of 32 voxels, word (z, y, xw) at
// (z * Y + y) * W32 + xw, so a region's rows are the words with xw = its
// region column.  One warp handles one region per level (lane l holds rows
// l*RPL .. l*RPL+RPL-1, row rho = z_local * TY + y_local); all levels run in
// one cooperative launch with a grid barrier per level.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <vector>

#include <cooperative_groups.h>

#include "mf_internal.cuh"

namespace mf {

namespace cg = cooperative_groups;
typedef unsigned int u32;

// masks M[d][word] bit b = [c_f(v -> v + D(d)) > 0] and T[word] bit b = [c_f(v,t) > 0]
// (a warp per grid row z * Y + y, lanes over x: coalesced plane reads, no
// 64-bit index division)
__device__ __forceinline__ void glr3d_mask_row(const Geom &g, const DevState &st, int W32, u32 *M, u32 *T, int row,
                                               int lane) {
    const size_t n = (size_t)g.n;
    const size_t nw = (size_t)g.Z * g.Y * W32;
    const size_t v0 = (size_t)row * g.X, w0 = (size_t)row * W32;
    for (int xw = 0; xw < W32; ++xw) {
        const int x = xw * 32 + lane;
        const bool in = x < g.X;
        const size_t v = v0 + x;
        int c[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) c[d] = in ? __ldg(&st.cap[d * n + v]) : 0;
        const int tc = in ? __ldg(&st.tcap[v]) : 0;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const unsigned m = __ballot_sync(0xffffffffu, c[d] > 0);
            if (lane == 0) M[d * nw + w0 + xw] = m;
        }
        const unsigned m = __ballot_sync(0xffffffffu, tc > 0);
        if (lane == 0) T[w0 + xw] = m;
    }
}

__global__ void glr3d_masks_kernel(const Geom g, const DevState st, int W32, u32 *M, u32 *T) {
    const int rows = g.Z * g.Y;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += nwarps)
        glr3d_mask_row(g, st, W32, M, T, row, threadIdx.x & 31);
}

template <int TY, int TZ>
struct Glr3 {
    // 16-row tiles: lanes 16..31 hold no row
    static constexpr int NR = TY * TZ, RPL = NR < 32 ? 1 : NR / 32, LZ = TY / RPL;
};

// One level for one region (a warp).  level 0 seeds from T; level l > 0 from
// S_{l-1} and the inter-region arcs into it.  Writes S_l; raises the labels
// of the vertices it adds.  Returns whether the region's set grew.
template <int TY, int TZ>
__device__ bool glr3d_region(const Geom &g, int W32, int r, const u32 *__restrict__ M, const u32 *__restrict__ T,
                             const u32 *Sin, u32 *Sout, int level, int *lab) {
    using C = Glr3<TY, TZ>;
    constexpr int RPL = C::RPL, LZ = C::LZ;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const size_t nw = (size_t)g.Z * g.Y * W32;
    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    u32 m[6][RPL], s[RPL], s0[RPL];
    size_t wi[RPL];
    bool rowin[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int rho = lane * RPL + j, yl = rho % TY, zl = rho / TY;
        const int y = ry * TY + yl, z = rz * TZ + zl;
        rowin[j] = rho < C::NR && y < g.Y && z < g.Z;
        wi[j] = ((size_t)z * g.Y + y) * W32 + rx;
        if (rowin[j]) {
#pragma unroll
            for (int d = 0; d < 6; ++d) m[d][j] = M[d * nw + wi[j]];
            s0[j] = level == 0 ? 0u : Sin[wi[j]];
            u32 sd = level == 0 ? T[wi[j]] : s0[j];
            if (level > 0) {
                // residual inter-region arcs into S_{l-1}
                if (rx > 0 && ((m[1][j] & 1u) && (Sin[wi[j] - 1] >> 31))) sd |= 1u;
                if (rx + 1 < g.RX && ((m[0][j] >> 31) && (Sin[wi[j] + 1] & 1u))) sd |= 1u << 31;
                if (yl == 0 && y > 0) sd |= m[3][j] & Sin[wi[j] - W32];
                if (yl == TY - 1 && y + 1 < g.Y) sd |= m[2][j] & Sin[wi[j] + W32];
                if (zl == 0 && z > 0) sd |= m[5][j] & Sin[wi[j] - (size_t)g.Y * W32];
                if (zl == TZ - 1 && z + 1 < g.Z) sd |= m[4][j] & Sin[wi[j] + (size_t)g.Y * W32];
            }
            s[j] = sd;
        } else {
#pragma unroll
            for (int d = 0; d < 6; ++d) m[d][j] = 0u;
            s0[j] = 0u;
            s[j] = 0u;
        }
    }
    // closure inside the region (arcs between rows of the tile, and along x within the word)
    for (;;) {
        const u32 up = __shfl_up_sync(FULL, s[RPL - 1], 1);
        const u32 dn = __shfl_down_sync(FULL, s[0], 1);
        bool any = false;
        u32 nf[RPL];
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int rho = lane * RPL + j, yl = rho % TY, zl = rho / TY;
            const u32 zm = __shfl_up_sync(FULL, s[j], LZ);
            const u32 zp = __shfl_down_sync(FULL, s[j], LZ);
            const u32 fa = j == 0 ? up : s[j - 1];
            const u32 fb = j == RPL - 1 ? dn : s[j + 1];
            u32 a = (m[0][j] & (s[j] >> 1)) | (m[1][j] & (s[j] << 1));
            if (yl < TY - 1) a |= m[2][j] & fb;
            if (yl > 0) a |= m[3][j] & fa;
            if (zl < TZ - 1) a |= m[4][j] & zp;
            if (zl > 0) a |= m[5][j] & zm;
            a &= ~s[j];
            // close whole x-runs at once (Kogge-Stone along the word)
            u32 pl = m[0][j] & ~s[j], pr = m[1][j] & ~s[j], f = a;
            {
                u32 q = f, p = pl;
                q |= p & (q >> 1);  p &= p >> 1;
                q |= p & (q >> 2);  p &= p >> 2;
                q |= p & (q >> 4);  p &= p >> 4;
                q |= p & (q >> 8);  p &= p >> 8;
                q |= p & (q >> 16);
                u32 b2 = f;
                p = pr;
                b2 |= p & (b2 << 1);  p &= p << 1;
                b2 |= p & (b2 << 2);  p &= p << 2;
                b2 |= p & (b2 << 4);  p &= p << 4;
                b2 |= p & (b2 << 8);  p &= p << 8;
                b2 |= p & (b2 << 16);
                f = q | b2;
            }
            nf[j] = f;
            any |= f != 0u;
        }
        if (!__any_sync(FULL, any)) break;
#pragma unroll
        for (int j = 0; j < RPL; ++j) s[j] |= nf[j];
    }
    bool grew = false;
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        if (!rowin[j]) continue;
        Sout[wi[j]] = s[j];
        u32 nwb = level == 0 ? 0u : (s[j] & ~s0[j]);
        grew |= nwb != 0u;
        if (!lab) continue;  // a plain closure: no labels
        const int rho = lane * RPL + j;
        const size_t row0 = ((size_t)(rz * TZ + rho / TY) * g.Y + (ry * TY + rho % TY)) * g.X + (size_t)rx * 32;
        for (; nwb; nwb &= nwb - 1) {
            int *p = &lab[row0 + __ffs((int)nwb) - 1];
            if (*p < level) *p = level;
        }
    }
    return __any_sync(FULL, grew);
}

// Per-region "grew at level l" flags (two bytes per region, by level parity):
// S_l(r) depends only on S_{l-1} of r and of its six neighbour regions, so a
// region none of which grew at level l-1 keeps its set at level l and is
// skipped.  Its level-l buffer then still holds S_{l-2}(r) = S_{l-1}(r) = S_l(r)
// (it did not grow at l-1 either); level 1 processes every region.
__device__ __forceinline__ bool region_or_nbr_grew(const Geom &g, const unsigned char *f, int r) {
    const int lane = threadIdx.x & 31;
    bool b = false;
    if (lane < 6) {
        const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
        const int qx = rx + arc_dx(6, lane), qy = ry + arc_dy(6, lane), qz = rz + arc_dz(6, lane);
        if (qx >= 0 && qx < g.RX && qy >= 0 && qy < g.RY && qz >= 0 && qz < g.RZ)
            b = f[(qz * g.RY + qy) * g.RX + qx] != 0;
    } else if (lane == 6) {
        b = f[r] != 0;
    }
    return __any_sync(0xffffffffu, b);
}

// the region flags follow the level sets in the relabel scratch
__host__ __device__ __forceinline__ unsigned char *glr3d_region_flags(u32 *B, size_t words) {
    return (unsigned char *)(B + words);
}

// all levels in one cooperative launch; flags[3] triple-buffered "grew" words
template <int TY, int TZ>
__global__ void glr3d_levels_kernel(const Geom g, int W32, const u32 *__restrict__ M, const u32 *__restrict__ T,
                                    u32 *A, u32 *B, int *lab, int *flags, int *levels_out, int max_levels) {
    cg::grid_group grid = cg::this_grid();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int r = wid; r < g.nreg; r += nwarps) glr3d_region<TY, TZ>(g, W32, r, M, T, nullptr, B, 0, lab);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flags[1] = 0;
        flags[2] = 0;
    }
    grid.sync();
    unsigned char *chg = glr3d_region_flags(B, (size_t)g.Z * g.Y * W32);
    int level = 1;
    for (; level < max_levels; ++level) {
        const u32 *in = (level & 1) ? B : A;
        u32 *out = (level & 1) ? A : B;
        const unsigned char *cin = chg + (size_t)((level - 1) & 1) * g.nreg;
        unsigned char *cout = chg + (size_t)(level & 1) * g.nreg;
        bool grew = false;
        for (int r = wid; r < g.nreg; r += nwarps) {
            bool gr = false;
            if (level == 1 || region_or_nbr_grew(g, cin, r)) gr = glr3d_region<TY, TZ>(g, W32, r, M, T, in, out, level, lab);
            if (lane == 0) cout[r] = gr;
            grew |= gr;
        }
        if (grew && lane == 0) atomicOr(&flags[level % 3], 1);
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(level + 1) % 3] = 0;
        grid.sync();
        if (!*(volatile int *)&flags[level % 3]) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *levels_out = level + 1;
}

// The finish over grid rows [row0, row1) (row = z * Y + y) of the set S, a
// warp per row and lanes over x (tiles are 32 voxels wide: the 32 voxels of
// a word lie in one region): unreached vertices get d_inf, a region holding
// excess below d_inf becomes active, and the labels of boundary vertices (an
// in-grid neighbour in another region) go to the histogram, bins below SB
// into the block's shared copy sh, equal labels of a warp as one update.
__device__ __forceinline__ void glr3d_finish_rows(const Geom &g, const DevState &st, int W32, const u32 *S, int row0,
                                                  int row1, int *sh, int SB) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int row = row0 + (int)(threadIdx.x >> 5); row < row1; row += nw) {
        const int z = row / g.Y, y = row - z * g.Y;
        const int ly = y & (g.ty - 1), lz = z & (g.tz - 1);
        const bool yzb = (ly == 0 && y > 0) || (ly == g.ty - 1 && y + 1 < g.Y) || (lz == 0 && z > 0) ||
                         (lz == g.tz - 1 && z + 1 < g.Z);
        const int rbase = ((z >> g.sz) * g.RY + (y >> g.sy)) * g.RX;
        const size_t v0 = (size_t)row * g.X;
        for (int xw = 0; xw < W32; ++xw) {
            const int x = xw * 32 + lane;
            const u32 sw = S[(size_t)row * W32 + xw];
            int l = g.dinf, e = 0;
            if (x < g.X) {
                l = st.lab[v0 + x];
                e = st.exc[v0 + x];
                if (!((sw >> lane) & 1u) && l != g.dinf) {
                    l = g.dinf;
                    st.lab[v0 + x] = l;
                }
            }
            const bool live = l < g.dinf;
            if (__any_sync(0xffffffffu, live && e > 0) && lane == 0) st.active[rbase + xw] = 1;
            const bool xb = (lane == 0 && x > 0) || (lane == 31 && x + 1 < g.X);
            const int key = live && (xb || yzb) ? l : -1;
            const unsigned mm = __match_any_sync(0xffffffffu, key);
            if (key >= 0 && lane == __ffs(mm) - 1) {
                const int c = __popc(mm);
                if (key < SB) atomicAdd(&sh[key], c);
                else atomicAdd(&st.hist[key < kHistBins ? key : kHistBins], c);
            }
        }
    }
}

// unreached vertices get d_inf; boundary-label histogram and region activity
__global__ void glr3d_finish_kernel(const Geom g, const DevState st, int W32, const u32 *A, const u32 *B) {
    constexpr int SB = 2048;
    // the set of the last level run (levels = st.ctr[kGlrLevels]): level 0
    // and the even levels write B, the odd levels A
    const int last = st.ctr[kGlrLevels] - 1;
    const u32 *S = (last % 2 == 1) ? A : B;
    __shared__ int sh[SB];
    for (int b = threadIdx.x; b < SB; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const int rows = g.Z * g.Y;
    const int per = (rows + gridDim.x - 1) / gridDim.x;  // a block takes a run of rows
    const int r0 = blockIdx.x * per;
    glr3d_finish_rows(g, st, W32, S, r0, min(rows, r0 + per), sh, SB);
    __syncthreads();
    for (int b = threadIdx.x; b < SB; b += blockDim.x)
        if (sh[b]) atomicAdd(&st.hist[b], sh[b]);
}

__global__ void glr3d_count_kernel(const DevState st, int nreg) {
    int c = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) c += st.active[r] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st.ctr[kActiveRegions], c);
}

// ---- cut extraction (Sec. 2) on the same masks --------------------------------
// S_min = closure of {e > 0} under residual arcs, S_max = V minus {v -> t}.
// Both as pull closures: v joins when its masked arc of some direction d
// leads to a member.  which = 0 (S_min): the bit of d at v is [c_f(v + D(d)
// -> v) > 0] (the arc into v), seeds e > 0; which = 1 ({v -> t}): the bit is
// [c_f(v -> v + D(d)) > 0], seeds c_f(v,t) > 0.
__device__ __forceinline__ void cut3d_masks_range(const Geom &g, const DevState &st, int W32, int which, u32 *M,
                                                  u32 *S, size_t t, size_t end, size_t step) {
    const size_t n = (size_t)g.n;
    const size_t words = (size_t)g.Z * g.Y * W32;
    // t and end differ from a multiple of 32 by the lane only, so a warp stays converged
    for (; t < end; t += step) {
        const size_t w = t >> 5;
        const int xw = (int)(w % W32), y = (int)((w / W32) % g.Y), z = (int)(w / ((size_t)W32 * g.Y));
        const int x = xw * 32 + (int)(t & 31);
        const bool in = x < g.X;
        const size_t v = ((size_t)z * g.Y + y) * g.X + x;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            bool b = false;
            if (in) {
                if (which == 1) {
                    b = st.cap[d * n + v] > 0;
                } else {
                    const int wx = x + arc_dx(6, d), wy = y + arc_dy(6, d), wz = z + arc_dz(6, d);
                    if (wx >= 0 && wx < g.X && wy >= 0 && wy < g.Y && wz >= 0 && wz < g.Z)
                        b = st.cap[(d ^ 1) * n + ((size_t)wz * g.Y + wy) * g.X + wx] > 0;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, b);
            if ((threadIdx.x & 31) == 0) M[d * words + w] = m;
        }
        const unsigned m = __ballot_sync(0xffffffffu, in && (which == 1 ? st.tcap[v] > 0 : st.exc[v] > 0));
        if ((threadIdx.x & 31) == 0) S[w] = m;
    }
}

__global__ void cut3d_masks_kernel(const Geom g, const DevState st, int W32, int which, u32 *M, u32 *S) {
    const size_t words = (size_t)g.Z * g.Y * W32;
    cut3d_masks_range(g, st, W32, which, M, S, blockIdx.x * (size_t)blockDim.x + threadIdx.x, words * 32,
                      (size_t)gridDim.x * blockDim.x);
}

// passes over all regions (a warp each: seeds across the faces from the
// current set, closure inside) until a pass adds nothing; the set grows in
// place, which only speeds up the fixed point
template <int TY, int TZ>
__global__ void closure3d_kernel(const Geom g, int W32, const u32 *__restrict__ M, u32 *S, int *flags,
                                 int *passes_out, int max_passes) {
    cg::grid_group grid = cg::this_grid();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flags[1] = 0;
        flags[2] = 0;
    }
    grid.sync();
    int pass = 1;  // the words of passes 1 and 2 were cleared above; pass p clears those of p + 1
    for (; pass <= max_passes; ++pass) {
        bool grew = false;
        for (int r = wid; r < g.nreg; r += nwarps)
            grew |= glr3d_region<TY, TZ>(g, W32, r, M, nullptr, S, S, 1, nullptr);
        if (grew && lane == 0) atomicOr(&flags[pass % 3], 1);
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(pass + 1) % 3] = 0;
        grid.sync();
        if (!*(volatile int *)&flags[pass % 3]) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *passes_out = pass;
}

__global__ void cut3d_bytes_kernel(const Geom g, int W32, const u32 *Smin, const u32 *Tset, unsigned char *smin,
                                   unsigned char *smax) {
    const int lane = threadIdx.x & 31;
    const int rows = g.Z * g.Y;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows; row += nwarps) {
        const size_t v0 = (size_t)row * g.X, w0 = (size_t)row * W32;
        for (int xw = 0; xw < W32; ++xw) {
            const int x = xw * 32 + lane;
            if (x >= g.X) continue;
            smin[v0 + x] = (unsigned char)((Smin[w0 + xw] >> lane) & 1u);
            smax[v0 + x] = (unsigned char)(1u - ((Tset[w0 + xw] >> lane) & 1u));
        }
    }
}

template <int TY, int TZ>
static cudaError_t cut3d_impl(const Geom &g, const DevState &st, void *scratch, unsigned char *smin,
                              unsigned char *smax, int *h_passes, cudaStream_t s) {
    const int W32 = (g.X + 31) / 32;
    const size_t words = (size_t)g.Z * g.Y * W32;
    u32 *M = (u32 *)scratch;
    u32 *Smin = M + 6 * words;
    u32 *Tset = Smin + words;
    const int mb = (int)std::min<size_t>((words * 32 + 255) / 256, device_sms() * 32);
    int max_blocks = 0;
    {
        const cudaError_t e_mb = coop_max_blocks((const void *)closure3d_kernel<TY, TZ>, 256, 0, &max_blocks);
        if (e_mb != cudaSuccess) return e_mb;
    }
    const int nblocks = std::min((g.nreg + 7) / 8, max_blocks);
    for (int which = 0; which < 2; ++which) {
        u32 *S = which == 0 ? Smin : Tset;
        cut3d_masks_kernel<<<mb, 256, 0, s>>>(g, st, W32, which, M, S);
        Geom gg = g;
        int w32 = W32, max_passes = 1 << 20;
        const u32 *pm = M;
        u32 *ps = S;
        int *flags = &st.ctr[kGlrFlags], *cnt = &st.ctr[kGlrLevels];
        void *args[] = {&gg, &w32, (void *)&pm, &ps, &flags, &cnt, &max_passes};
        cudaError_t e = cudaLaunchCooperativeKernel((const void *)closure3d_kernel<TY, TZ>, dim3(nblocks), dim3(256),
                                                    args, 0, s);
        // closure passes made, copied without waiting (h_passes is pinned host memory)
        if (e == cudaSuccess && h_passes) e = cudaMemcpyAsync(h_passes + which, cnt, 4, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
    }
    const int nb = (int)std::min<size_t>(((size_t)g.n + 255) / 256, device_sms() * 32);
    cut3d_bytes_kernel<<<nb, 256, 0, s>>>(g, W32, Smin, Tset, smin, smax);
    return cudaGetLastError();
}

cudaError_t cut3d(const Geom &g, const DevState &st, void *scratch, unsigned char *smin, unsigned char *smax,
                  int *h_passes, cudaStream_t s) {
    if (g.ty == 16 && g.tz == 8) return cut3d_impl<16, 8>(g, st, scratch, smin, smax, h_passes, s);
    if (g.ty == 8 && g.tz == 8) return cut3d_impl<8, 8>(g, st, scratch, smin, smax, h_passes, s);
    if (g.ty == 8 && g.tz == 4) return cut3d_impl<8, 4>(g, st, scratch, smin, smax, h_passes, s);
    if (g.ty == 4 && g.tz == 4) return cut3d_impl<4, 4>(g, st, scratch, smin, smax, h_passes, s);
    if (g.ty == 8 && g.tz == 2) return cut3d_impl<8, 2>(g, st, scratch, smin, smax, h_passes, s);
    return cudaErrorInvalidValue;
}

// ---- the same relabel for many 3D grids at once (batched solves) -------------
// As glr2d_batch: one launch builds the masks of every due grid, one
// cooperative launch runs their levels, a work unit is (grid, region), a warp
// per unit; then one finish launch over (grid, chunk) units and one count.
// The masks keep the layout above; the job's A/B fields hold the grid's level
// sets (u32 words here).
template <int TY, int TZ>
__device__ __forceinline__ bool glr3d_unit(const GlrJob2 &J, int r, const u32 *in, u32 *out, int level) {
    const size_t words = (size_t)J.g.Z * J.g.Y * J.W64;
    const u32 *M = (const u32 *)J.M;
    const u32 *T = M + 6 * words;
    return glr3d_region<TY, TZ>(J.g, J.W64, r, M, T, in, out, level, J.st.lab);
}

__device__ __forceinline__ bool glr3d_unit_any(const GlrJob2 &J, int r, const u32 *in, u32 *out, int level) {
    if (J.g.ty == 16) return glr3d_unit<16, 8>(J, r, in, out, level);
    if (J.g.tz == 8) return glr3d_unit<8, 8>(J, r, in, out, level);
    if (J.g.ty == 4) return glr3d_unit<4, 4>(J, r, in, out, level);
    if (J.g.tz == 2) return glr3d_unit<8, 2>(J, r, in, out, level);
    return glr3d_unit<8, 4>(J, r, in, out, level);
}

__global__ void glr3d_batch_levels_kernel(const GlrJob2 *__restrict__ jobs, int njobs, const int *__restrict__ unit_job,
                                          int nunits, int *any, int max_levels) {
    cg::grid_group grid = cg::this_grid();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int u = wid; u < nunits; u += nwarps) {
        const GlrJob2 &J = jobs[unit_job[u]];
        glr3d_unit_any(J, u - J.unit0, nullptr, (u32 *)J.B, 0);
    }
    if (blockIdx.x == 0) {
        for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
            jobs[j].st.ctr[kGlrFlags + 1] = 0;
            jobs[j].st.ctr[kGlrFlags + 2] = 0;
        }
        if (threadIdx.x == 0) any[1] = any[2] = 0;
    }
    grid.sync();
    int level = 1;
    for (; level < max_levels; ++level) {
        const int f = level % 3, fp = (level + 2) % 3;
        bool grew_any = false;
        for (int u = wid; u < nunits; u += nwarps) {
            const GlrJob2 &J = jobs[unit_job[u]];
            if (level > 1 && !*(volatile int *)&J.st.ctr[kGlrFlags + fp]) continue;  // stopped growing
            const u32 *in = (const u32 *)((level & 1) ? J.B : J.A);
            u32 *out = (u32 *)((level & 1) ? J.A : J.B);
            const int r = u - J.unit0;
            unsigned char *chg = glr3d_region_flags((u32 *)J.B, (size_t)J.g.Z * J.g.Y * J.W64);
            bool grew = false;
            if (level == 1 || region_or_nbr_grew(J.g, chg + (size_t)((level - 1) & 1) * J.g.nreg, r))
                grew = glr3d_unit_any(J, r, in, out, level);
            if (lane == 0) chg[(size_t)(level & 1) * J.g.nreg + r] = grew;
            if (grew && lane == 0) atomicOr(&J.st.ctr[kGlrFlags + f], 1);
            grew_any |= grew;
        }
        if (grew_any && lane == 0) atomicOr(&any[f], 1);
        if (blockIdx.x == 0) {
            for (int j = threadIdx.x; j < njobs; j += blockDim.x) jobs[j].st.ctr[kGlrFlags + (level + 1) % 3] = 0;
            if (threadIdx.x == 0) any[(level + 1) % 3] = 0;
        }
        grid.sync();
        if (blockIdx.x == 0) {
            for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
                const int *c = jobs[j].st.ctr;
                const bool ran = level == 1 || *(volatile const int *)&c[kGlrFlags + fp];
                if (ran && !*(volatile const int *)&c[kGlrFlags + f]) jobs[j].st.ctr[kGlrLevels] = level + 1;
            }
        }
        if (!*(volatile int *)&any[f]) break;
    }
    if (level >= max_levels && blockIdx.x == 0)
        for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
            const int *c = jobs[j].st.ctr;
            if (*(volatile const int *)&c[kGlrFlags + (level + 2) % 3]) jobs[j].st.ctr[kGlrLevels] = level;
        }
}

__global__ void glr3d_batch_reset_kernel(const GlrJob2 *__restrict__ jobs) {
    const DevState &st = jobs[blockIdx.x].st;
    const int nreg = jobs[blockIdx.x].g.nreg;
    for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x) st.hist[b] = 0;
    for (int r = threadIdx.x; r < nreg; r += blockDim.x) st.active[r] = 0;
    if (threadIdx.x == 0) st.ctr[kActiveRegions] = 0;
}

constexpr int kFinishChunk3 = 16384;  // voxels per unit of the batched cut bytes
constexpr int kFinishRows3 = 64;      // grid rows per unit of the batched finish
__global__ void glr3d_batch_finish_kernel(const GlrJob2 *__restrict__ jobs, const int2 *__restrict__ chunks, int nchunks) {
    constexpr int SB = 2048;
    __shared__ int sh[SB];
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int2 w = chunks[c];
        const GlrJob2 &J = jobs[w.x];
        const Geom &g = J.g;
        const DevState &st = J.st;
        for (int b = threadIdx.x; b < SB; b += blockDim.x) sh[b] = 0;
        __syncthreads();
        const int last = st.ctr[kGlrLevels] - 1;
        const u32 *S = (const u32 *)((last % 2 == 1) ? J.A : J.B);
        const int r0 = w.y * kFinishRows3;
        glr3d_finish_rows(g, st, J.W64, S, r0, min(g.Z * g.Y, r0 + kFinishRows3), sh, SB);
        __syncthreads();
        for (int b = threadIdx.x; b < SB; b += blockDim.x)
            if (sh[b]) atomicAdd(&st.hist[b], sh[b]);
        __syncthreads();
    }
}

__global__ void glr3d_batch_count_kernel(const GlrJob2 *__restrict__ jobs) {
    const DevState &st = jobs[blockIdx.x].st;
    const int nreg = jobs[blockIdx.x].g.nreg;
    int c = 0;
    for (int r = threadIdx.x; r < nreg; r += blockDim.x) c += st.active[r] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st.ctr[kActiveRegions], c);
}

// The relabel masks of many grids in one launch: a block per unit (grid,
// kMaskRows rows z * Y + y), a warp per row.
__global__ void glr3d_masks_batch_kernel(const GlrJob2 *__restrict__ jobs, const int2 *__restrict__ rows, int nrows) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int u = blockIdx.x; u < nrows; u += gridDim.x) {
        const int2 r = rows[u];
        const GlrJob2 &J = jobs[r.x];
        const size_t words = (size_t)J.g.Z * J.g.Y * J.W64;
        u32 *M = (u32 *)J.M;
        const int y0 = r.y * kMaskRows, y1 = min(J.g.Z * J.g.Y, y0 + kMaskRows);
        for (int row = y0 + warp; row < y1; row += nw)
            glr3d_mask_row(J.g, J.st, J.W64, M, M + 6 * words, row, threadIdx.x & 31);
    }
}

// The cut masks and seeds of many grids in one launch, a block per unit (grid,
// kMaskRows rows); which as in cut3d_masks_kernel, the seeds go to set A
// (which = 0) or B (which = 1).
__global__ void cut3d_masks_batch_kernel(const GlrJob2 *__restrict__ jobs, const int2 *__restrict__ rows, int nrows,
                                         int which) {
    for (int u = blockIdx.x; u < nrows; u += gridDim.x) {
        const int2 r = rows[u];
        const GlrJob2 &J = jobs[r.x];
        const int y0 = r.y * kMaskRows, y1 = min(J.g.Z * J.g.Y, y0 + kMaskRows);
        const size_t t0 = (size_t)y0 * J.W64 * 32 + threadIdx.x, end = (size_t)y1 * J.W64 * 32;
        cut3d_masks_range(J.g, J.st, J.W64, which, (u32 *)J.M, (u32 *)(which == 0 ? J.A : J.B), t0, end,
                          blockDim.x);
    }
}

static void push_mask_rows3(std::vector<int2> &rows, int job, int nrow) {
    for (int c = 0; c < (nrow + kMaskRows - 1) / kMaskRows; ++c) rows.push_back(make_int2(job, c));
}

cudaError_t glr3d_batch(const std::vector<GlrJob2> &jobs_in, GlrBatchBufs &bb, cudaStream_t s) {
    const int njobs = (int)jobs_in.size();
    if (njobs == 0) return cudaSuccess;
    std::vector<GlrJob2> jobs(jobs_in);
    std::vector<int> unit_job;
    std::vector<int2> chunks, rows;
    for (int j = 0; j < njobs; ++j) {
        GlrJob2 &J = jobs[j];
        J.W64 = (J.g.X + 31) / 32;  // here: 32-voxel words per row
        J.BY = 0;
        const size_t words = (size_t)J.g.Z * J.g.Y * J.W64;
        u32 *M = (u32 *)J.scratch;
        J.M = (unsigned long long *)M;
        J.A = (unsigned long long *)(M + 7 * words);
        J.B = (unsigned long long *)(M + 8 * words);
        J.unit0 = (int)unit_job.size();
        for (int r = 0; r < J.g.nreg; ++r) unit_job.push_back(j);
        const int nc = (int)((J.g.Z * J.g.Y + kFinishRows3 - 1) / kFinishRows3);
        for (int c = 0; c < nc; ++c) chunks.push_back(make_int2(j, c));
        push_mask_rows3(rows, j, J.g.Z * J.g.Y);
    }
    cudaError_t e = bb.reserve(njobs * sizeof(GlrJob2), unit_job.size() * sizeof(int), chunks.size() * sizeof(int2));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(bb.jobs, jobs.data(), njobs * sizeof(GlrJob2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bb.units, unit_job.data(), unit_job.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bb.chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = bb.upload_rows(rows, s);
    if (e != cudaSuccess) return e;
    const int nrows = (int)rows.size();
    glr3d_masks_batch_kernel<<<std::min(nrows, device_sms() * 8), 256, 0, s>>>((const GlrJob2 *)bb.jobs,
                                                                               (const int2 *)bb.rows, nrows);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int max_blocks = 0;
    e = coop_max_blocks((const void *)glr3d_batch_levels_kernel, 256, 0, &max_blocks);
    if (e != cudaSuccess) return e;
    const int nunits = (int)unit_job.size();
    const int nblocks = std::max(1, std::min((nunits + 7) / 8, max_blocks));
    const GlrJob2 *pj = (const GlrJob2 *)bb.jobs;
    const int *pu = (const int *)bb.units;
    int *pany = bb.any;
    int nj = njobs, nu = nunits, ml = 1 << 20;
    void *args[] = {(void *)&pj, &nj, (void *)&pu, &nu, &pany, &ml};
    e = cudaLaunchCooperativeKernel((const void *)glr3d_batch_levels_kernel, dim3(nblocks), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    glr3d_batch_reset_kernel<<<njobs, 256, 0, s>>>(pj);
    const int nch = (int)chunks.size();
    glr3d_batch_finish_kernel<<<std::min(nch, device_sms() * 8), 256, 0, s>>>(pj, (const int2 *)bb.chunks, nch);
    glr3d_batch_count_kernel<<<njobs, 256, 0, s>>>(pj);
    e = cudaGetLastError();
    return e == cudaSuccess ? glr_batch_out(pj, njobs, 0, s) : e;
}

// ---- both cut closures of many 3D grids at once (batched solves) --------------
__global__ void cut3d_batch_closure_kernel(const GlrJob2 *__restrict__ jobs, int njobs, const int *__restrict__ unit_job,
                                           int nunits, int *any, int max_passes, int which) {
    cg::grid_group grid = cg::this_grid();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0) {
        for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
            jobs[j].st.ctr[kGlrFlags + 1] = 0;
            jobs[j].st.ctr[kGlrFlags + 2] = 0;
        }
        if (threadIdx.x == 0) any[1] = any[2] = 0;
    }
    grid.sync();
    int pass = 1;
    for (; pass <= max_passes; ++pass) {
        const int f = pass % 3, fp = (pass + 2) % 3;
        bool grew_any = false;
        for (int u = wid; u < nunits; u += nwarps) {
            const GlrJob2 &J = jobs[unit_job[u]];
            if (pass > 1 && !*(volatile int *)&J.st.ctr[kGlrFlags + fp]) continue;  // closed
            u32 *S = (u32 *)(which == 0 ? J.A : J.B);
            const u32 *M = (const u32 *)J.M;
            const int r = u - J.unit0;
            bool grew;
            if (J.g.ty == 16) grew = glr3d_region<16, 8>(J.g, J.W64, r, M, nullptr, S, S, 1, nullptr);
            else if (J.g.tz == 8) grew = glr3d_region<8, 8>(J.g, J.W64, r, M, nullptr, S, S, 1, nullptr);
            else if (J.g.ty == 4) grew = glr3d_region<4, 4>(J.g, J.W64, r, M, nullptr, S, S, 1, nullptr);
            else if (J.g.tz == 2) grew = glr3d_region<8, 2>(J.g, J.W64, r, M, nullptr, S, S, 1, nullptr);
            else grew = glr3d_region<8, 4>(J.g, J.W64, r, M, nullptr, S, S, 1, nullptr);
            if (grew && lane == 0) atomicOr(&J.st.ctr[kGlrFlags + f], 1);
            grew_any |= grew;
        }
        if (grew_any && lane == 0) atomicOr(&any[f], 1);
        if (blockIdx.x == 0) {
            for (int j = threadIdx.x; j < njobs; j += blockDim.x) jobs[j].st.ctr[kGlrFlags + (pass + 1) % 3] = 0;
            if (threadIdx.x == 0) any[(pass + 1) % 3] = 0;
        }
        grid.sync();
        if (blockIdx.x == 0) {
            for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
                const int *c = jobs[j].st.ctr;
                const bool ran = pass == 1 || *(volatile const int *)&c[kGlrFlags + fp];
                if (ran && !*(volatile const int *)&c[kGlrFlags + f]) jobs[j].st.ctr[kGlrLevels] = pass;
            }
        }
        if (!*(volatile int *)&any[f]) break;
    }
}

__global__ void cut3d_batch_bytes_kernel(const GlrJob2 *__restrict__ jobs, const int2 *__restrict__ chunks, int nchunks) {
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int2 w = chunks[c];
        const GlrJob2 &J = jobs[w.x];
        const Geom &g = J.g;
        const u32 *Smin = (const u32 *)J.A, *Tset = (const u32 *)J.B;
        const size_t v0 = (size_t)w.y * kFinishChunk3, v1 = min((size_t)g.n, v0 + kFinishChunk3);
        for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            const int x = (int)(v % g.X), y = (int)((v / g.X) % g.Y), z = (int)(v / ((size_t)g.X * g.Y));
            const size_t wd = ((size_t)z * g.Y + y) * J.W64 + (x >> 5);
            J.smin[v] = (Smin[wd] >> (x & 31)) & 1u;
            J.smax[v] = !((Tset[wd] >> (x & 31)) & 1u);
        }
    }
}

cudaError_t cut3d_batch(const std::vector<GlrJob2> &jobs_in, GlrBatchBufs &bb, cudaStream_t s) {
    const int njobs = (int)jobs_in.size();
    if (njobs == 0) return cudaSuccess;
    std::vector<GlrJob2> jobs(jobs_in);
    std::vector<int> unit_job;
    std::vector<int2> chunks, rows;
    for (int j = 0; j < njobs; ++j) {
        GlrJob2 &J = jobs[j];
        J.W64 = (J.g.X + 31) / 32;
        J.BY = 0;
        const size_t words = (size_t)J.g.Z * J.g.Y * J.W64;
        u32 *M = (u32 *)J.scratch;
        J.M = (unsigned long long *)M;
        J.A = (unsigned long long *)(M + 6 * words);  // S_min (the layout of cut3d)
        J.B = (unsigned long long *)(M + 7 * words);  // the set {v -> t}
        J.unit0 = (int)unit_job.size();
        for (int r = 0; r < J.g.nreg; ++r) unit_job.push_back(j);
        const int nc = (int)((J.g.n + kFinishChunk3 - 1) / kFinishChunk3);
        for (int c = 0; c < nc; ++c) chunks.push_back(make_int2(j, c));
        push_mask_rows3(rows, j, J.g.Z * J.g.Y);
    }
    cudaError_t e = bb.reserve(njobs * sizeof(GlrJob2), unit_job.size() * sizeof(int), chunks.size() * sizeof(int2));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(bb.jobs, jobs.data(), njobs * sizeof(GlrJob2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bb.units, unit_job.data(), unit_job.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bb.chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = bb.upload_rows(rows, s);
    if (e != cudaSuccess) return e;
    const int nrows = (int)rows.size();
    int max_blocks = 0;
    e = coop_max_blocks((const void *)cut3d_batch_closure_kernel, 256, 0, &max_blocks);
    if (e != cudaSuccess) return e;
    const int nunits = (int)unit_job.size();
    const int nblocks = std::max(1, std::min((nunits + 7) / 8, max_blocks));
    for (int which = 0; which < 2; ++which) {
        cut3d_masks_batch_kernel<<<std::min(nrows, device_sms() * 8), 256, 0, s>>>(
            (const GlrJob2 *)bb.jobs, (const int2 *)bb.rows, nrows, which);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const GlrJob2 *pj = (const GlrJob2 *)bb.jobs;
        const int *pu = (const int *)bb.units;
        int *pany = bb.any;
        int nj = njobs, nu = nunits, mp = 1 << 20, wh = which;
        void *args[] = {(void *)&pj, &nj, (void *)&pu, &nu, &pany, &mp, &wh};
        e = cudaLaunchCooperativeKernel((const void *)cut3d_batch_closure_kernel, dim3(nblocks), dim3(256), args, 0, s);
        if (e == cudaSuccess) e = glr_batch_out(pj, njobs, which, s);
        if (e != cudaSuccess) return e;
    }
    const int nch = (int)chunks.size();
    cut3d_batch_bytes_kernel<<<std::min(nch, device_sms() * 8), 256, 0, s>>>((const GlrJob2 *)bb.jobs,
                                                                            (const int2 *)bb.chunks, nch);
    return cudaGetLastError();
}

bool glr3d_supported(const Geom &g) {
    return g.tx == 32 && g.tz > 1 && ((g.ty == 16 && g.tz == 8) || (g.ty == 8 && g.tz == 8) || (g.ty == 8 && g.tz == 4) ||
                                      (g.ty == 4 && g.tz == 4) || (g.ty == 8 && g.tz == 2));
}

size_t glr3d_scratch_bytes(const Geom &g) {
    const size_t words = (size_t)g.Z * g.Y * ((g.X + 31) / 32);
    return words * 4 * (6 + 1 + 2) + 2 * (size_t)g.nreg;  // masks, T, two level sets, region flags
}

template <int TY, int TZ>
static cudaError_t glr3d_impl(const Geom &g, const DevState &st, void *scratch, cudaStream_t s) {
    const int W32 = (g.X + 31) / 32;
    const size_t words = (size_t)g.Z * g.Y * W32;
    u32 *M = (u32 *)scratch;
    u32 *T = M + 6 * words;
    u32 *A = T + words;
    u32 *B = A + words;
    const int mb = (int)std::min<size_t>(((size_t)g.Z * g.Y + 7) / 8, device_sms() * 32);
    glr3d_masks_kernel<<<mb, 256, 0, s>>>(g, st, W32, M, T);
    int max_blocks = 0;
    {
        const cudaError_t e_mb = coop_max_blocks((const void *)glr3d_levels_kernel<TY, TZ>, 256, 0, &max_blocks);
        if (e_mb != cudaSuccess) return e_mb;
    }
    const int nblocks = std::min((g.nreg + 7) / 8, max_blocks);
    int *flags = &st.ctr[kGlrFlags];
    int *lvl = &st.ctr[kGlrLevels];
    int max_levels = 1 << 20;
    Geom gg = g;
    int w32 = W32;
    const u32 *pm = M, *pt = T;
    u32 *pa = A, *pb = B;
    int *lab = st.lab;
    void *args[] = {&gg, &w32, (void *)&pm, (void *)&pt, &pa, &pb, &lab, &flags, &lvl, &max_levels};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)glr3d_levels_kernel<TY, TZ>, dim3(nblocks), dim3(256),
                                                args, 0, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(st.hist, 0, (kHistBins + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.active, 0, (size_t)g.nreg, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st.ctr[kActiveRegions], 0, 4, s);
    if (e != cudaSuccess) return e;
    const int nb = (int)std::min<size_t>(((size_t)g.Z * g.Y + 7) / 8, device_sms() * 32);
    glr3d_finish_kernel<<<nb, 256, 0, s>>>(g, st, W32, A, B);
    glr3d_count_kernel<<<(g.nreg + 255) / 256, 256, 0, s>>>(st, g.nreg);
    return cudaGetLastError();
}

cudaError_t glr3d(const Geom &g, const DevState &st, void *scratch, cudaStream_t s) {
    if (g.ty == 16 && g.tz == 8) return glr3d_impl<16, 8>(g, st, scratch, s);
    if (g.ty == 8 && g.tz == 8) return glr3d_impl<8, 8>(g, st, scratch, s);
    if (g.ty == 8 && g.tz == 4) return glr3d_impl<8, 4>(g, st, scratch, s);
    if (g.ty == 4 && g.tz == 4) return glr3d_impl<4, 4>(g, st, scratch, s);
    if (g.ty == 8 && g.tz == 2) return glr3d_impl<8, 2>(g, st, scratch, s);
    return cudaErrorInvalidValue;
}

}  // namespace mf
