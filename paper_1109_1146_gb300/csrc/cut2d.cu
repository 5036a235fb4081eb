// Cut extraction for 2D grids on bit masks.
//
// After the last sweep the preflow is maximum (Sec. 2: {v : e(v) > 0} does
// not reach t).  The two canonical minimum cuts are residual closures:
//   S_min = vertices reachable from {e > 0} over residual arcs,
//   S_max = complement of {v : v -> t}.
// Both are computed as "pull" closures: a vertex joins the set when one of
// its masked arcs leads into the set.  For {v -> t} the mask of direction d at
// v is [c_f(v -> v+D(d)) > 0]; for the forward closure S_min the mask is
// [c_f(v+D(d) -> v) > 0] (the arc into v from its d-neighbour), which turns
// forward reachability into the same pull rule.
//
// The grid is cut into 64x64 blocks (independent of the region tiling); one
// warp floods one block on 64-bit row words (lane = two rows) until it is
// closed, using the set bits of the neighbouring blocks read at the start of
// the pass; passes repeat until no block changes.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cooperative_groups.h>

#include "mf_internal.cuh"

namespace mf {

namespace cg = cooperative_groups;
typedef unsigned long long u64;

// Build the masks: M[d][y][w] bit b (x = 64w + b) and the seed words S[y][w].
// which = 0: forward masks (arc into v) and seeds e > 0; which = 1: arc out of
// v and seeds c_f(v,t) > 0.
template <int CONN>
__device__ __forceinline__ void cut_masks_range(const Geom &g, const DevState &st, int W64, int which, unsigned *M,
                                                unsigned *S, size_t t, size_t end, size_t step) {
    const size_t n = (size_t)g.n;
    const size_t rowbits = (size_t)W64 * 64;
    const size_t plane32 = (size_t)g.Y * W64 * 2;
    // t and end differ from a multiple of 32 by the lane only, so a warp stays converged
    for (; t < end; t += step) {
        const int y = (int)(t / rowbits), x = (int)(t % rowbits);
        const bool in = x < g.X;
        const size_t v = (size_t)y * g.X + x;
        const size_t word32 = t >> 5;  // rows are whole 64-bit words, so t/32 indexes u32 halves
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            bool b = false;
            if (in) {
                if (which == 1) {
                    b = st.cap[d * n + v] > 0;
                } else {
                    const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d);
                    if (wx >= 0 && wx < g.X && wy >= 0 && wy < g.Y)
                        b = st.cap[(d ^ 1) * n + (size_t)wy * g.X + wx] > 0;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, b);
            if ((threadIdx.x & 31) == 0) M[d * plane32 + word32] = m;
        }
        const bool s = in && (which == 1 ? st.tcap[v] > 0 : st.exc[v] > 0);
        const unsigned m = __ballot_sync(0xffffffffu, s);
        if ((threadIdx.x & 31) == 0) S[word32] = m;
    }
}

template <int CONN>
__global__ void cut_masks_kernel(const Geom g, const DevState st, int W64, int which, unsigned *M,
                                 unsigned *S) {
    cut_masks_range<CONN>(g, st, W64, which, M, S, blockIdx.x * (size_t)blockDim.x + threadIdx.x,
                          (size_t)W64 * 64 * g.Y, (size_t)gridDim.x * blockDim.x);
}

__device__ __forceinline__ u64 fill_row(u64 g, u64 pl, u64 pr) {
    u64 a = g, p = pl;
    a |= p & (a >> 1);  p &= p >> 1;
    a |= p & (a >> 2);  p &= p >> 2;
    a |= p & (a >> 4);  p &= p >> 4;
    a |= p & (a >> 8);  p &= p >> 8;
    a |= p & (a >> 16); p &= p >> 16;
    a |= p & (a >> 32);
    u64 b = g;
    p = pr;
    b |= p & (b << 1);  p &= p << 1;
    b |= p & (b << 2);  p &= p << 2;
    b |= p & (b << 4);  p &= p << 4;
    b |= p & (b << 8);  p &= p << 8;
    b |= p & (b << 16); p &= p << 16;
    b |= p & (b << 32);
    return a | b;
}

// One 64x64 block closes its part of the set (one warp, in place); returns
// whether it grew.
template <int CONN>
__device__ bool cut_block2d(const Geom &g, int W64, int blk, const u64 *__restrict__ M, u64 *S) {
    const int lane = threadIdx.x & 31;
    const int bx = blk % W64, by = blk / W64;
    const size_t plane = (size_t)g.Y * W64;
    auto word = [&](const u64 *A, int y, int w) -> u64 {
        return (y >= 0 && y < g.Y && w >= 0 && w < W64) ? A[(size_t)y * W64 + w] : 0ull;
    };
    u64 s[2], m[CONN][2], sl[2], sr[2], s0[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int y = by * 64 + 2 * lane + j;
        s[j] = word(S, y, bx);
        s0[j] = s[j];
        sl[j] = word(S, y, bx - 1) >> 63;       // x = 64bx - 1
        sr[j] = word(S, y, bx + 1) & 1ull;      // x = 64bx + 64
#pragma unroll
        for (int d = 0; d < CONN; ++d) m[d][j] = word(M + d * plane, y, bx);
    }
    // rows just outside the block (lane 0: above, lane 31: below)
    const int ya = by * 64 - 1, yb = by * 64 + 64;
    const u64 sa = word(S, ya, bx), sal = word(S, ya, bx - 1) >> 63, sar = word(S, ya, bx + 1) & 1ull;
    const u64 sb = word(S, yb, bx), sbl = word(S, yb, bx - 1) >> 63, sbr = word(S, yb, bx + 1) & 1ull;
    bool grew = false;
    for (;;) {
        // neighbour rows with their outside bits
        const u64 up = __shfl_up_sync(0xffffffffu, s[1], 1), upl = __shfl_up_sync(0xffffffffu, sl[1], 1),
                  upr = __shfl_up_sync(0xffffffffu, sr[1], 1);
        const u64 dn = __shfl_down_sync(0xffffffffu, s[0], 1), dnl = __shfl_down_sync(0xffffffffu, sl[0], 1),
                  dnr = __shfl_down_sync(0xffffffffu, sr[0], 1);
        bool any = false;
        u64 nf[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const u64 fa = j == 0 ? (lane == 0 ? sa : up) : s[0];
            const u64 fal = j == 0 ? (lane == 0 ? sal : upl) : sl[0];
            const u64 far_ = j == 0 ? (lane == 0 ? sar : upr) : sr[0];
            const u64 fb = j == 1 ? (lane == 31 ? sb : dn) : s[1];
            const u64 fbl = j == 1 ? (lane == 31 ? sbl : dnl) : sl[1];
            const u64 fbr = j == 1 ? (lane == 31 ? sbr : dnr) : sr[1];
            u64 a = (m[0][j] & ((s[j] >> 1) | (sr[j] << 63))) | (m[1][j] & ((s[j] << 1) | sl[j])) |
                    (m[2][j] & fb) | (m[3][j] & fa);
            if (CONN == 8)
                a |= (m[4][j] & ((fb >> 1) | (fbr << 63))) | (m[5][j] & ((fa << 1) | fal)) |
                     (m[6][j] & ((fb << 1) | fbl)) | (m[7][j] & ((fa >> 1) | (far_ << 63)));
            a &= ~s[j];
            a = fill_row(a, m[0][j] & ~s[j], m[1][j] & ~s[j]);
            nf[j] = a;
            any |= a != 0ull;
        }
        if (!__any_sync(0xffffffffu, any)) break;
        grew = true;
#pragma unroll
        for (int j = 0; j < 2; ++j) s[j] |= nf[j];
    }
    if (grew) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int y = by * 64 + 2 * lane + j;
            if (y < g.Y && s[j] != s0[j]) S[(size_t)y * W64 + bx] = s[j];
        }
    }
    return grew;
}

// Passes over all blocks (a warp each) until a pass adds nothing, in one
// cooperative launch; flags[3] triple-buffered "grew" words as in the relabel.
template <int CONN>
__global__ void cut_closure2d_kernel(const Geom g, int W64, int BY, const u64 *__restrict__ M, u64 *S, int *flags,
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
        for (int b = wid; b < W64 * BY; b += nwarps) grew |= cut_block2d<CONN>(g, W64, b, M, S);
        if (grew && lane == 0) atomicOr(&flags[pass % 3], 1);
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(pass + 1) % 3] = 0;
        grid.sync();
        if (!*(volatile int *)&flags[pass % 3]) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *passes_out = pass;
}

// S_min / S_max bytes from the two closures
__global__ void cut_bytes_kernel(const Geom g, int W64, const u64 *Smin, const u64 *Tset, unsigned char *smin,
                                 unsigned char *smax) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < (size_t)g.n; v += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(v / g.X), x = (int)(v % g.X);
        const size_t w = (size_t)y * W64 + (x >> 6);
        smin[v] = (Smin[w] >> (x & 63)) & 1ull;
        smax[v] = !((Tset[w] >> (x & 63)) & 1ull);
    }
}

// ---- global relabel (exact region distance) on the same bit masks ---------------
//
// The region distance of Sec. 4.1 counts the inter-region arcs of a path to
// t (labels may only drop across them).  Level sets by a 0-1 BFS:
//   S_0     = vertices that reach t inside their own region;
//   S_{k}   = intra-region closure of S_{k-1} plus the vertices with a residual
//             inter-region arc into S_{k-1}.
// A vertex first found at level k has region distance k; vertices never found
// cannot reach t (distance d_inf).  The labeling is raised to max(d, level),
// which keeps it valid (a maximum of two valid labelings is valid, Sec. 6.1)
// and monotone.  One launch per level; the set is double-buffered so a level
// reads only the previous level.

// bits of a row word whose arc in direction (dx, dy) stays inside the region tile
__device__ __forceinline__ u64 intra_bits(const Geom &g, int y, int dx, int dy) {
    u64 m = ~0ull;
    if (dx > 0) m &= g.tx == 64 ? 0x7fffffffffffffffull : 0x7fffffff7fffffffull;
    if (dx < 0) m &= g.tx == 64 ? 0xfffffffffffffffeull : 0xfffffffefffffffeull;
    if (dy > 0 && ((y + 1) & (g.ty - 1)) == 0) m = 0;
    if (dy < 0 && (y & (g.ty - 1)) == 0) m = 0;
    return m;
}

template <int CONN>
struct GlrBlock {
    int bx, by, yy[2];
    u64 m[CONN][2], mi[CONN][2];  // residual masks of the block rows; intra-region part
};

template <int CONN>
__device__ __forceinline__ void glr_load_block(const Geom &g, int W64, int blk, const u64 *__restrict__ M,
                                               GlrBlock<CONN> &B) {
    const int lane = threadIdx.x & 31;
    const size_t plane = (size_t)g.Y * W64;
    B.bx = blk % W64;
    B.by = blk / W64;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int y = B.by * 64 + 2 * lane + j;
        B.yy[j] = y;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            B.m[d][j] = y < g.Y ? M[d * plane + (size_t)y * W64 + B.bx] : 0ull;
            B.mi[d][j] = B.m[d][j] & intra_bits(g, y, arc_dx(CONN, d), arc_dy(CONN, d));
        }
    }
}

template <int CONN>
__device__ __forceinline__ bool glr_level_block(const Geom &g, int W64, const GlrBlock<CONN> &B,
                                                const u64 *__restrict__ Sin, u64 *Sout, int level, int *lab) {
    const int lane = threadIdx.x & 31;
    const int bx = B.bx, by = B.by;
    auto word = [&](const u64 *A, int y, int w) -> u64 {
        return (y >= 0 && y < g.Y && w >= 0 && w < W64) ? A[(size_t)y * W64 + w] : 0ull;
    };
    const auto &m = B.m;
    const auto &mi = B.mi;
    const int *yy = B.yy;
    u64 s[2], s0[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        s[j] = word(Sin, yy[j], bx);
        s0[j] = s[j];
    }
    if (level > 0) {
        // vertices with a residual inter-region arc into S_{level-1}
        u64 sl[2], sr[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            sl[j] = word(Sin, yy[j], bx - 1) >> 63;
            sr[j] = word(Sin, yy[j], bx + 1) & 1ull;
        }
        const int ya = by * 64 - 1, yb = by * 64 + 64;
        const u64 sa = word(Sin, ya, bx), sal = word(Sin, ya, bx - 1) >> 63, sar = word(Sin, ya, bx + 1) & 1ull;
        const u64 sb = word(Sin, yb, bx), sbl = word(Sin, yb, bx - 1) >> 63, sbr = word(Sin, yb, bx + 1) & 1ull;
        const u64 up = __shfl_up_sync(0xffffffffu, s[1], 1), upl = __shfl_up_sync(0xffffffffu, sl[1], 1),
                  upr = __shfl_up_sync(0xffffffffu, sr[1], 1);
        const u64 dn = __shfl_down_sync(0xffffffffu, s[0], 1), dnl = __shfl_down_sync(0xffffffffu, sl[0], 1),
                  dnr = __shfl_down_sync(0xffffffffu, sr[0], 1);
        u64 nf[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const u64 fa = j == 0 ? (lane == 0 ? sa : up) : s[0];
            const u64 fal = j == 0 ? (lane == 0 ? sal : upl) : sl[0];
            const u64 far_ = j == 0 ? (lane == 0 ? sar : upr) : sr[0];
            const u64 fb = j == 1 ? (lane == 31 ? sb : dn) : s[1];
            const u64 fbl = j == 1 ? (lane == 31 ? sbl : dnl) : sl[1];
            const u64 fbr = j == 1 ? (lane == 31 ? sbr : dnr) : sr[1];
            u64 c[8];
            c[0] = (s[j] >> 1) | (sr[j] << 63);
            c[1] = (s[j] << 1) | sl[j];
            c[2] = fb;
            c[3] = fa;
            c[4] = (fb >> 1) | (fbr << 63);
            c[5] = (fa << 1) | fal;
            c[6] = (fb << 1) | fbl;
            c[7] = (fa >> 1) | (far_ << 63);
            u64 a = 0;
#pragma unroll
            for (int d = 0; d < CONN; ++d) a |= (m[d][j] & ~mi[d][j]) & c[d];
            nf[j] = a & ~s[j];
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) s[j] |= nf[j];
    }
    // closure inside the regions (intra-region arcs only)
    for (;;) {
        const u64 up = __shfl_up_sync(0xffffffffu, s[1], 1);
        const u64 dn = __shfl_down_sync(0xffffffffu, s[0], 1);
        bool any = false;
        u64 nf[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const u64 fa = j == 0 ? (lane == 0 ? 0ull : up) : s[0];
            const u64 fb = j == 1 ? (lane == 31 ? 0ull : dn) : s[1];
            u64 a = (mi[0][j] & (s[j] >> 1)) | (mi[1][j] & (s[j] << 1)) | (mi[2][j] & fb) | (mi[3][j] & fa);
            if (CONN == 8)
                a |= (mi[4][j] & (fb >> 1)) | (mi[5][j] & (fa << 1)) | (mi[6][j] & (fb << 1)) | (mi[7][j] & (fa >> 1));
            a &= ~s[j];
            a = fill_row(a, mi[0][j] & ~s[j], mi[1][j] & ~s[j]);
            nf[j] = a;
            any |= a != 0ull;
        }
        if (!__any_sync(0xffffffffu, any)) break;
#pragma unroll
        for (int j = 0; j < 2; ++j) s[j] |= nf[j];
    }
    bool grew = false;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        if (yy[j] >= g.Y) continue;
        Sout[(size_t)yy[j] * W64 + bx] = s[j];
        // members found at this level get label max(d, level); level 0 changes nothing
        u64 nw = level == 0 ? 0ull : (s[j] & ~s0[j]);
        grew |= nw != 0ull;
        for (; nw; nw &= nw - 1) {
            const int x = bx * 64 + __ffsll((long long)nw) - 1;
            int *p = &lab[(size_t)yy[j] * g.X + x];
            if (*p < level) *p = level;
        }
    }
    return __any_sync(0xffffffffu, grew);
}

// All levels in one cooperative launch: every warp takes 64x64 blocks in turn,
// and the grid synchronises between levels.  flags[3] are "a block grew"
// words, triple-buffered so that the word read after level L is not reset
// before every thread has passed the next grid barrier.
template <int CONN>
__global__ void glr_levels_kernel(const Geom g, int W64, int BY, const u64 *__restrict__ M, u64 *A, u64 *B,
                                  int *lab, int *flags, int *levels_out, int max_levels) {
    cg::grid_group grid = cg::this_grid();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int nblk = W64 * BY;
    const bool resident = nblk <= nwarps;  // each warp keeps its block's masks in registers
    GlrBlock<CONN> blkm;
    if (resident && wid < nblk) glr_load_block<CONN>(g, W64, wid, M, blkm);
    for (int b = wid; b < nblk; b += nwarps) {
        if (!resident) glr_load_block<CONN>(g, W64, b, M, blkm);
        glr_level_block<CONN>(g, W64, blkm, A, B, 0, lab);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flags[1] = 0;
        flags[2] = 0;
    }
    grid.sync();
    int level = 1;
    for (; level < max_levels; ++level) {
        const u64 *in = (level & 1) ? B : A;
        u64 *out = (level & 1) ? A : B;
        bool grew = false;
        for (int b = wid; b < nblk; b += nwarps) {
            if (!resident) glr_load_block<CONN>(g, W64, b, M, blkm);
            grew |= glr_level_block<CONN>(g, W64, blkm, in, out, level, lab);
        }
        if (grew && lane == 0) atomicOr(&flags[level % 3], 1);
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(level + 1) % 3] = 0;
        grid.sync();
        if (!*(volatile int *)&flags[level % 3]) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *levels_out = level + 1;
}

// After the last level: unreached vertices get d_inf; rebuild the boundary-label
// histogram (per-block shared counts for small labels, merged once) and mark
// the regions that still hold an active vertex.
template <int CONN>
__global__ void glr_finish_kernel(const Geom g, const DevState st, int W64, const u64 *A, const u64 *B) {
    constexpr int SB = 2048;  // labels below SB are counted in shared memory first
    // the set of the last level run (levels = st.ctr[kGlrLevels]): level 0
    // and the even levels write B, the odd levels A
    const int last = st.ctr[kGlrLevels] - 1;
    const u64 *S = (last % 2 == 1) ? A : B;
    __shared__ int sh[SB];
    for (int b = threadIdx.x; b < SB; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < (size_t)g.n; v += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(v / g.X), x = (int)(v % g.X);
        int l = st.lab[v];
        if (!((S[(size_t)y * W64 + (x >> 6)] >> (x & 63)) & 1ull)) {
            l = g.dinf;
            st.lab[v] = l;
        }
        if (l >= g.dinf) continue;
        const int r = ((y >> g.sy) * g.RX) + (x >> g.sx);
        if (st.exc[v] > 0) st.active[r] = 1;
        const int lx = x & (g.tx - 1), ly = y & (g.ty - 1);
        if (lx != 0 && lx != g.tx - 1 && ly != 0 && ly != g.ty - 1) continue;  // tile interior: not in B
        bool inB = false;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d);
            if (wx < 0 || wx >= g.X || wy < 0 || wy >= g.Y) continue;
            if (((wy >> g.sy) * g.RX + (wx >> g.sx)) != r) inB = true;
        }
        if (!inB) continue;
        if (l < SB) atomicAdd(&sh[l], 1);
        else atomicAdd(&st.hist[l < kHistBins ? l : kHistBins], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < SB; b += blockDim.x)
        if (sh[b]) atomicAdd(&st.hist[b], sh[b]);
}

__global__ void count_active_kernel(const DevState st, int nreg) {
    int c = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) c += st.active[r] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st.ctr[kActiveRegions], c);
}

// Exact region-distance relabel of a 2D grid (tiles 32 or 64 wide).  Uses the
// cut scratch (masks and two set buffers).  levels: number of BFS levels run.
template <int CONN>
static cudaError_t glr2d_impl(const Geom &g, const DevState &st, void *scratch, cudaStream_t s) {
    const int W64 = (g.X + 63) / 64, BY = (g.Y + 63) / 64;
    const size_t plane = (size_t)g.Y * W64;
    u64 *M = (u64 *)scratch;
    u64 *A = M + CONN * plane;
    u64 *B = A + plane;
    const size_t total = (size_t)W64 * 64 * g.Y;
    const int mb = (int)std::min<size_t>((total + 255) / 256, device_sms() * 32);
    cut_masks_kernel<CONN><<<mb, 256, 0, s>>>(g, st, W64, 1, (unsigned *)M, (unsigned *)A);
    // one cooperative launch for all levels; the grid must be co-resident
    int max_blocks = 0;
    {
        const cudaError_t e_mb = coop_max_blocks((const void *)glr_levels_kernel<CONN>, 256, 0, &max_blocks);
        if (e_mb != cudaSuccess) return e_mb;
    }
    int nblocks = std::min((W64 * BY + 7) / 8, max_blocks);
    int *flags = &st.ctr[kGlrFlags];
    int *lvl = &st.ctr[kGlrLevels];
    int max_levels = 1 << 20;
    u64 *pa = A, *pb = B;
    int *lab = st.lab;
    Geom gg = g;
    int w64 = W64, by = BY;
    void *args[] = {&gg, &w64, &by, (void *)&M, &pa, &pb, &lab, &flags, &lvl, &max_levels};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)glr_levels_kernel<CONN>, dim3(nblocks), dim3(256),
                                                args, 0, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(st.hist, 0, (kHistBins + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.active, 0, (size_t)g.nreg, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st.ctr[kActiveRegions], 0, 4, s);
    if (e != cudaSuccess) return e;
    const int nb = (int)std::min<size_t>(((size_t)g.n + 255) / 256, device_sms() * 32);
    glr_finish_kernel<CONN><<<nb, 256, 0, s>>>(g, st, W64, A, B);
    count_active_kernel<<<(g.nreg + 255) / 256, 256, 0, s>>>(st, g.nreg);
    return cudaGetLastError();
}

// ---- the same relabel for many 2D grids at once (batched solves) -------------
// One cooperative launch runs the levels of every grid of a batch that is due
// for a relabel: a work unit is (grid, 64x64 block), a warp takes units in
// turn, the grid barrier separates levels.  A grid whose set did not grow at
// a level has its final set and is skipped from then on; its level count is
// recorded when it stops.  The masks before the levels, the finish (d_inf for
// unreached vertices, the boundary-label histogram, region activity) and the
// count of active regions after them are one launch each over all grids.
template <int CONN>
__device__ __forceinline__ bool glr2d_unit(const GlrJob2 &J, int blk, const u64 *in, u64 *out, int level) {
    GlrBlock<CONN> B;
    glr_load_block<CONN>(J.g, J.W64, blk, J.M, B);
    return glr_level_block<CONN>(J.g, J.W64, B, in, out, level, J.st.lab);
}

__global__ void glr2d_batch_levels_kernel(const GlrJob2 *__restrict__ jobs, int njobs, const int *__restrict__ unit_job,
                                          int nunits, int *any, int max_levels) {
    cg::grid_group grid = cg::this_grid();
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int u = wid; u < nunits; u += nwarps) {
        const GlrJob2 &J = jobs[unit_job[u]];
        const int blk = u - J.unit0;
        if (J.conn == 4) glr2d_unit<4>(J, blk, J.A, J.B, 0);
        else glr2d_unit<8>(J, blk, J.A, J.B, 0);
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
        const int f = level % 3, fp = (level + 2) % 3;  // this level's words, the previous level's
        bool grew_any = false;
        for (int u = wid; u < nunits; u += nwarps) {
            const int j = unit_job[u];
            const GlrJob2 &J = jobs[j];
            if (level > 1 && !*(volatile int *)&J.st.ctr[kGlrFlags + fp]) continue;  // stopped growing
            const u64 *in = (level & 1) ? J.B : J.A;
            u64 *out = (level & 1) ? J.A : J.B;
            const bool grew = J.conn == 4 ? glr2d_unit<4>(J, u - J.unit0, in, out, level)
                                          : glr2d_unit<8>(J, u - J.unit0, in, out, level);
            if (grew && lane == 0) atomicOr(&J.st.ctr[kGlrFlags + f], 1);
            grew_any |= grew;
        }
        if (grew_any && lane == 0) atomicOr(&any[f], 1);
        if (blockIdx.x == 0) {
            for (int j = threadIdx.x; j < njobs; j += blockDim.x) jobs[j].st.ctr[kGlrFlags + (level + 1) % 3] = 0;
            if (threadIdx.x == 0) any[(level + 1) % 3] = 0;
        }
        grid.sync();
        // a grid that ran this level and did not grow ends here: its sets of
        // this level and the previous one are equal
        if (blockIdx.x == 0) {
            for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
                const int *c = jobs[j].st.ctr;
                const bool ran = level == 1 || *(volatile const int *)&c[kGlrFlags + fp];
                if (ran && !*(volatile const int *)&c[kGlrFlags + f]) jobs[j].st.ctr[kGlrLevels] = level + 1;
            }
        }
        if (!*(volatile int *)&any[f]) break;
    }
    if (level >= max_levels && blockIdx.x == 0)  // still growing at the cap: their last level is level - 1
        for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
            const int *c = jobs[j].st.ctr;
            if (*(volatile const int *)&c[kGlrFlags + (level + 2) % 3]) jobs[j].st.ctr[kGlrLevels] = level;
        }
}

// per grid (one block each): clear its histogram, region activity and active count
__global__ void glr_batch_reset_kernel(const GlrJob2 *__restrict__ jobs) {
    const DevState &st = jobs[blockIdx.x].st;
    const int nreg = jobs[blockIdx.x].g.nreg;
    for (int b = threadIdx.x; b <= kHistBins; b += blockDim.x) st.hist[b] = 0;
    for (int r = threadIdx.x; r < nreg; r += blockDim.x) st.active[r] = 0;
    if (threadIdx.x == 0) st.ctr[kActiveRegions] = 0;
}

// the finish of every grid: a block per (grid, chunk of 16384 vertices)
constexpr int kFinishChunk = 16384;
template <int CONN>
__device__ __forceinline__ void glr2d_finish_chunk(const GlrJob2 &J, size_t v0, size_t v1, int *sh, int SB) {
    const Geom &g = J.g;
    const DevState &st = J.st;
    const int last = st.ctr[kGlrLevels] - 1;
    const u64 *S = (last % 2 == 1) ? J.A : J.B;
    for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const int y = (int)(v / g.X), x = (int)(v % g.X);
        int l = st.lab[v];
        if (!((S[(size_t)y * J.W64 + (x >> 6)] >> (x & 63)) & 1ull)) {
            l = g.dinf;
            st.lab[v] = l;
        }
        if (l >= g.dinf) continue;
        const int r = ((y >> g.sy) * g.RX) + (x >> g.sx);
        if (st.exc[v] > 0) st.active[r] = 1;
        const int lx = x & (g.tx - 1), ly = y & (g.ty - 1);
        if (lx != 0 && lx != g.tx - 1 && ly != 0 && ly != g.ty - 1) continue;
        bool inB = false;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d);
            if (wx < 0 || wx >= g.X || wy < 0 || wy >= g.Y) continue;
            if (((wy >> g.sy) * g.RX + (wx >> g.sx)) != r) inB = true;
        }
        if (!inB) continue;
        if (l < SB) atomicAdd(&sh[l], 1);
        else atomicAdd(&st.hist[l < kHistBins ? l : kHistBins], 1);
    }
}

__global__ void glr2d_batch_finish_kernel(const GlrJob2 *__restrict__ jobs, const int2 *__restrict__ chunks, int nchunks) {
    constexpr int SB = 2048;
    __shared__ int sh[SB];
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int2 w = chunks[c];
        const GlrJob2 &J = jobs[w.x];
        for (int b = threadIdx.x; b < SB; b += blockDim.x) sh[b] = 0;
        __syncthreads();
        const size_t v0 = (size_t)w.y * kFinishChunk, v1 = min((size_t)J.g.n, v0 + kFinishChunk);
        if (J.conn == 4) glr2d_finish_chunk<4>(J, v0, v1, sh, SB);
        else glr2d_finish_chunk<8>(J, v0, v1, sh, SB);
        __syncthreads();
        for (int b = threadIdx.x; b < SB; b += blockDim.x)
            if (sh[b]) atomicAdd(&J.st.hist[b], sh[b]);
        __syncthreads();
    }
}

// per grid (one block each): count its active regions
__global__ void glr_batch_count_kernel(const GlrJob2 *__restrict__ jobs) {
    const DevState &st = jobs[blockIdx.x].st;
    const int nreg = jobs[blockIdx.x].g.nreg;
    int c = 0;
    for (int r = threadIdx.x; r < nreg; r += blockDim.x) c += st.active[r] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st.ctr[kActiveRegions], c);
}

// The masks and seeds of many grids in one launch: a block per unit (grid,
// kMaskRows rows); which as in cut_masks_kernel, the seeds go to the grid's
// set A (set_b = 0) or B (set_b = 1).
__global__ void cut_masks_batch_kernel(const GlrJob2 *__restrict__ jobs, const int2 *__restrict__ rows, int nrows,
                                       int which, int set_b) {
    for (int u = blockIdx.x; u < nrows; u += gridDim.x) {
        const int2 r = rows[u];
        const GlrJob2 &J = jobs[r.x];
        const size_t rowbits = (size_t)J.W64 * 64;
        const int y0 = r.y * kMaskRows, y1 = min(J.g.Y, y0 + kMaskRows);
        unsigned *S = (unsigned *)(set_b ? J.B : J.A);
        const size_t t0 = (size_t)y0 * rowbits + threadIdx.x, end = (size_t)y1 * rowbits;
        if (J.conn == 4) cut_masks_range<4>(J.g, J.st, J.W64, which, (unsigned *)J.M, S, t0, end, blockDim.x);
        else cut_masks_range<8>(J.g, J.st, J.W64, which, (unsigned *)J.M, S, t0, end, blockDim.x);
    }
}

static void push_mask_rows(std::vector<int2> &rows, int job, int nrow) {
    for (int c = 0; c < (nrow + kMaskRows - 1) / kMaskRows; ++c) rows.push_back(make_int2(job, c));
}

cudaError_t glr2d_batch(const std::vector<GlrJob2> &jobs_in, GlrBatchBufs &bb, cudaStream_t s) {
    const int njobs = (int)jobs_in.size();
    if (njobs == 0) return cudaSuccess;
    std::vector<GlrJob2> jobs(jobs_in);
    std::vector<int> unit_job;
    std::vector<int2> chunks, rows;
    for (int j = 0; j < njobs; ++j) {
        GlrJob2 &J = jobs[j];
        J.W64 = (J.g.X + 63) / 64;
        J.BY = (J.g.Y + 63) / 64;
        const size_t plane = (size_t)J.g.Y * J.W64;
        J.M = (u64 *)J.scratch;
        J.A = J.M + J.conn * plane;
        J.B = J.A + plane;
        J.unit0 = (int)unit_job.size();
        for (int b = 0; b < J.W64 * J.BY; ++b) unit_job.push_back(j);
        const int nc = (int)((J.g.n + kFinishChunk - 1) / kFinishChunk);
        for (int c = 0; c < nc; ++c) chunks.push_back(make_int2(j, c));
        push_mask_rows(rows, j, J.g.Y);
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
    // residual masks and the level-0 seeds of every grid
    const int nrows = (int)rows.size();
    cut_masks_batch_kernel<<<std::min(nrows, device_sms() * 8), 256, 0, s>>>((const GlrJob2 *)bb.jobs,
                                                                             (const int2 *)bb.rows, nrows, 1, 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int max_blocks = 0;
    e = coop_max_blocks((const void *)glr2d_batch_levels_kernel, 256, 0, &max_blocks);
    if (e != cudaSuccess) return e;
    const int nunits = (int)unit_job.size();
    const int nblocks = std::max(1, std::min((nunits + 7) / 8, max_blocks));
    const GlrJob2 *pj = (const GlrJob2 *)bb.jobs;
    const int *pu = (const int *)bb.units;
    int *pany = bb.any;
    int nj = njobs, nu = nunits, ml = 1 << 20;
    void *args[] = {(void *)&pj, &nj, (void *)&pu, &nu, &pany, &ml};
    e = cudaLaunchCooperativeKernel((const void *)glr2d_batch_levels_kernel, dim3(nblocks), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    glr_batch_reset_kernel<<<njobs, 256, 0, s>>>(pj);
    const int nch = (int)chunks.size();
    glr2d_batch_finish_kernel<<<std::min(nch, device_sms() * 8), 256, 0, s>>>(pj, (const int2 *)bb.chunks, nch);
    glr_batch_count_kernel<<<njobs, 256, 0, s>>>(pj);
    e = cudaGetLastError();
    return e == cudaSuccess ? glr_batch_out(pj, njobs, 0, s) : e;
}

// ---- both cut closures of many 2D grids at once (batched solves) --------------
// Per closure: the masks of every grid (one launch), then one cooperative
// launch of block passes over the units (grid, 64x64 block) of all grids, a
// grid leaving the passes once a pass adds nothing to its set; then the bytes
// of S_min and S_max of every grid in one launch.  The pass count of each
// closure lands in the grid's st.ctr[kGlrLevels].
__global__ void cut2d_batch_closure_kernel(const GlrJob2 *__restrict__ jobs, int njobs, const int *__restrict__ unit_job,
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
            u64 *S = which == 0 ? J.A : J.B;
            const bool grew = J.conn == 4 ? cut_block2d<4>(J.g, J.W64, u - J.unit0, J.M, S)
                                          : cut_block2d<8>(J.g, J.W64, u - J.unit0, J.M, S);
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

__global__ void cut2d_batch_bytes_kernel(const GlrJob2 *__restrict__ jobs, const int2 *__restrict__ chunks, int nchunks) {
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int2 w = chunks[c];
        const GlrJob2 &J = jobs[w.x];
        const size_t v0 = (size_t)w.y * kFinishChunk, v1 = min((size_t)J.g.n, v0 + kFinishChunk);
        for (size_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            const int y = (int)(v / J.g.X), x = (int)(v % J.g.X);
            const size_t wd = (size_t)y * J.W64 + (x >> 6);
            J.smin[v] = (J.A[wd] >> (x & 63)) & 1ull;
            J.smax[v] = !((J.B[wd] >> (x & 63)) & 1ull);
        }
    }
}

cudaError_t cut2d_batch(const std::vector<GlrJob2> &jobs_in, GlrBatchBufs &bb, cudaStream_t s) {
    const int njobs = (int)jobs_in.size();
    if (njobs == 0) return cudaSuccess;
    std::vector<GlrJob2> jobs(jobs_in);
    std::vector<int> unit_job;
    std::vector<int2> chunks, rows;
    for (int j = 0; j < njobs; ++j) {
        GlrJob2 &J = jobs[j];
        J.W64 = (J.g.X + 63) / 64;
        J.BY = (J.g.Y + 63) / 64;
        const size_t plane = (size_t)J.g.Y * J.W64;
        J.M = (u64 *)J.scratch;
        J.A = J.M + J.conn * plane;  // S_min
        J.B = J.A + plane;           // the set {v -> t}
        J.unit0 = (int)unit_job.size();
        for (int b = 0; b < J.W64 * J.BY; ++b) unit_job.push_back(j);
        const int nc = (int)((J.g.n + kFinishChunk - 1) / kFinishChunk);
        for (int c = 0; c < nc; ++c) chunks.push_back(make_int2(j, c));
        push_mask_rows(rows, j, J.g.Y);
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
    e = coop_max_blocks((const void *)cut2d_batch_closure_kernel, 256, 0, &max_blocks);
    if (e != cudaSuccess) return e;
    const int nunits = (int)unit_job.size();
    const int nblocks = std::max(1, std::min((nunits + 7) / 8, max_blocks));
    for (int which = 0; which < 2; ++which) {
        cut_masks_batch_kernel<<<std::min(nrows, device_sms() * 8), 256, 0, s>>>(
            (const GlrJob2 *)bb.jobs, (const int2 *)bb.rows, nrows, which, which);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const GlrJob2 *pj = (const GlrJob2 *)bb.jobs;
        const int *pu = (const int *)bb.units;
        int *pany = bb.any;
        int nj = njobs, nu = nunits, mp = 1 << 20, wh = which;
        void *args[] = {(void *)&pj, &nj, (void *)&pu, &nu, &pany, &mp, &wh};
        e = cudaLaunchCooperativeKernel((const void *)cut2d_batch_closure_kernel, dim3(nblocks), dim3(256), args, 0, s);
        if (e == cudaSuccess) e = glr_batch_out(pj, njobs, which, s);
        if (e != cudaSuccess) return e;
    }
    const int nch = (int)chunks.size();
    cut2d_batch_bytes_kernel<<<std::min(nch, device_sms() * 8), 256, 0, s>>>((const GlrJob2 *)bb.jobs,
                                                                            (const int2 *)bb.chunks, nch);
    return cudaGetLastError();
}

cudaError_t GlrBatchBufs::reserve(size_t jobs_bytes, size_t units_bytes, size_t chunks_bytes) {
    auto grow = [](void **p, size_t &cap, size_t want) -> cudaError_t {
        if (want <= cap) return cudaSuccess;
        if (*p) cudaFree(*p);
        *p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(p, want);
        if (e == cudaSuccess) cap = want;
        return e;
    };
    cudaError_t e = grow(&jobs, jobs_cap, jobs_bytes);
    if (e == cudaSuccess) e = grow(&units, units_cap, units_bytes);
    if (e == cudaSuccess) e = grow(&chunks, chunks_cap, chunks_bytes);
    if (e == cudaSuccess && !any) e = cudaMalloc(&any, 4 * sizeof(int));
    return e;
}

__global__ void glr_batch_out_kernel(const GlrJob2 *__restrict__ jobs, int njobs, int slot) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < njobs && jobs[j].hout) jobs[j].hout[slot] = jobs[j].st.ctr[kGlrLevels];
}

cudaError_t glr_batch_out(const GlrJob2 *jobs_dev, int njobs, int slot, cudaStream_t s) {
    if (njobs <= 0) return cudaSuccess;
    glr_batch_out_kernel<<<(njobs + 255) / 256, 256, 0, s>>>(jobs_dev, njobs, slot);
    return cudaGetLastError();
}

cudaError_t GlrBatchBufs::upload_rows(const std::vector<int2> &units_in, cudaStream_t s) {
    const size_t want = std::max<size_t>(1, units_in.size()) * sizeof(int2);
    if (want > rows_cap) {
        if (rows) cudaFree(rows);
        rows = nullptr;
        rows_cap = 0;
        const cudaError_t e = cudaMalloc(&rows, want);
        if (e != cudaSuccess) return e;
        rows_cap = want;
    }
    if (units_in.empty()) return cudaSuccess;
    return cudaMemcpyAsync(rows, units_in.data(), units_in.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
}

GlrBatchBufs::~GlrBatchBufs() {
    for (void *p : {jobs, units, chunks, rows, (void *)any})
        if (p) cudaFree(p);
}

bool glr2d_supported(const Geom &g) { return g.tz == 1 && g.Z == 1 && (g.tx == 64 || g.tx == 32); }

cudaError_t glr2d(int conn, const Geom &g, const DevState &st, void *scratch, cudaStream_t s) {
    if (conn == 4) return glr2d_impl<4>(g, st, scratch, s);
    if (conn == 8) return glr2d_impl<8>(g, st, scratch, s);
    return cudaErrorInvalidValue;
}

size_t cut2d_scratch_bytes(const Geom &g, int conn) {
    const size_t W64 = (size_t)(g.X + 63) / 64;
    return (size_t)(conn + 2) * g.Y * W64 * 8;  // masks + two sets
}

// Both closures; scratch must hold cut2d_scratch_bytes.  passes += passes made.
template <int CONN>
static cudaError_t cut2d_impl(const Geom &g, const DevState &st, void *scratch, unsigned char *smin,
                              unsigned char *smax, int *h_passes, cudaStream_t s) {
    const int W64 = (g.X + 63) / 64, BY = (g.Y + 63) / 64;
    const size_t plane = (size_t)g.Y * W64;
    u64 *M = (u64 *)scratch;
    u64 *Smin = M + CONN * plane;
    u64 *Tset = Smin + plane;
    const size_t total = (size_t)W64 * 64 * g.Y;
    const int mb = (int)std::min<size_t>((total + 255) / 256, device_sms() * 32);
    int max_blocks = 0;
    {
        const cudaError_t e_mb = coop_max_blocks((const void *)cut_closure2d_kernel<CONN>, 256, 0, &max_blocks);
        if (e_mb != cudaSuccess) return e_mb;
    }
    const int blocks = std::min((W64 * BY + 7) / 8, max_blocks);
    for (int which = 0; which < 2; ++which) {
        u64 *Sset = which == 0 ? Smin : Tset;
        cut_masks_kernel<CONN><<<mb, 256, 0, s>>>(g, st, W64, which, (unsigned *)M, (unsigned *)Sset);
        Geom gg = g;
        int w64 = W64, by = BY, max_passes = 1 << 20;
        const u64 *pm = M;
        u64 *ps = Sset;
        int *flags = &st.ctr[kGlrFlags], *cnt = &st.ctr[kGlrLevels];
        void *args[] = {&gg, &w64, &by, (void *)&pm, &ps, &flags, &cnt, &max_passes};
        cudaError_t e = cudaLaunchCooperativeKernel((const void *)cut_closure2d_kernel<CONN>, dim3(blocks), dim3(256),
                                                    args, 0, s);
        // closure passes made, copied without waiting (h_passes is pinned host memory)
        if (e == cudaSuccess && h_passes) e = cudaMemcpyAsync(h_passes + which, cnt, 4, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
    }
    const int nb = (int)std::min<size_t>(((size_t)g.n + 255) / 256, device_sms() * 32);
    cut_bytes_kernel<<<nb, 256, 0, s>>>(g, W64, Smin, Tset, smin, smax);
    return cudaGetLastError();
}

cudaError_t cut2d(int conn, const Geom &g, const DevState &st, void *scratch, unsigned char *smin,
                  unsigned char *smax, int *h_passes, cudaStream_t s) {
    if (conn == 4) return cut2d_impl<4>(g, st, scratch, smin, smax, h_passes, s);
    if (conn == 8) return cut2d_impl<8>(g, st, scratch, smin, smax, h_passes, s);
    return cudaErrorInvalidValue;
}

}  // namespace mf
