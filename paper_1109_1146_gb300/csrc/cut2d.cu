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

#include "mf_internal.cuh"

namespace mf {

typedef unsigned long long u64;

// Build the masks: M[d][y][w] bit b (x = 64w + b) and the seed words S[y][w].
// which = 0: forward masks (arc into v) and seeds e > 0; which = 1: arc out of
// v and seeds c_f(v,t) > 0.
template <int CONN>
__global__ void cut_masks_kernel(const Geom g, const DevState st, int W64, int which, unsigned *M,
                                 unsigned *S) {
    const size_t n = (size_t)g.n;
    const size_t rowbits = (size_t)W64 * 64;
    const size_t total = rowbits * g.Y;
    const size_t plane32 = (size_t)g.Y * W64 * 2;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
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

// One pass: every 64x64 block closes its part of the set (one warp per block).
template <int CONN>
__global__ void cut_pass2d_kernel(const Geom g, int W64, int BY, const u64 *__restrict__ M, u64 *S,
                                  int *changed) {
    const int lane = threadIdx.x & 31;
    const int blk = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (blk >= W64 * BY) return;
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
        if (lane == 0) *changed = 1;
    }
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

size_t cut2d_scratch_bytes(const Geom &g, int conn) {
    const size_t W64 = (size_t)(g.X + 63) / 64;
    return (size_t)(conn + 2) * g.Y * W64 * 8;  // masks + two sets
}

// Both closures; scratch must hold cut2d_scratch_bytes.  passes += passes made.
template <int CONN>
static cudaError_t cut2d_impl(const Geom &g, const DevState &st, void *scratch, unsigned char *smin,
                              unsigned char *smax, int *h_changed, int *passes, cudaStream_t s) {
    const int W64 = (g.X + 63) / 64, BY = (g.Y + 63) / 64;
    const size_t plane = (size_t)g.Y * W64;
    u64 *M = (u64 *)scratch;
    u64 *Smin = M + CONN * plane;
    u64 *Tset = Smin + plane;
    const size_t total = (size_t)W64 * 64 * g.Y;
    const int mb = (int)std::min<size_t>((total + 255) / 256, 152 * 32);
    const int blocks = (W64 * BY + 7) / 8;
    for (int which = 0; which < 2; ++which) {
        u64 *Sset = which == 0 ? Smin : Tset;
        cut_masks_kernel<CONN><<<mb, 256, 0, s>>>(g, st, W64, which, (unsigned *)M, (unsigned *)Sset);
        for (;;) {
            cudaError_t e = cudaMemsetAsync(&st.ctr[kChanged], 0, 4, s);
            if (e != cudaSuccess) return e;
            cut_pass2d_kernel<CONN><<<blocks, 256, 0, s>>>(g, W64, BY, M, Sset, &st.ctr[kChanged]);
            e = cudaMemcpyAsync(h_changed, &st.ctr[kChanged], 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            ++*passes;
            if (!*h_changed) break;
        }
    }
    const int nb = (int)std::min<size_t>(((size_t)g.n + 255) / 256, 152 * 32);
    cut_bytes_kernel<<<nb, 256, 0, s>>>(g, W64, Smin, Tset, smin, smax);
    return cudaGetLastError();
}

cudaError_t cut2d(int conn, const Geom &g, const DevState &st, void *scratch, unsigned char *smin,
                  unsigned char *smax, int *h_changed, int *passes, cudaStream_t s) {
    if (conn == 4) return cut2d_impl<4>(g, st, scratch, smin, smax, h_changed, passes, s);
    if (conn == 8) return cut2d_impl<8>(g, st, scratch, smin, smax, h_changed, passes, s);
    return cudaErrorInvalidValue;
}

}  // namespace mf
