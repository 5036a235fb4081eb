// Boundary-relabel heuristic (Sec. 6.1): a lower bound d' on the region
// distance computed from the boundary alone, then d := max(d, d').
//
// The auxiliary graph of the section has one node per (region, label) group of
// boundary vertices with d < d_inf, a length-0 arc from each group to the next
// higher label of its region (a valid labeling forbids paths inside a region
// from a higher label down to a lower one, so only upward reachability may be
// assumed) and a length-1 arc along every residual arc between two regions.
// d' of a group is its distance to the groups of label 0.
//
// Because of the length-0 chain, the groups of a region that lie within
// distance k of label 0 are exactly those with label <= L_k(R), a per-region
// threshold (L_0 = 0).  The search therefore keeps one threshold per region
// and advances all of them level by level:
//   L_{k+1}(R) = max(L_k(R), max over neighbour regions Q of
//                    max{ d(u) : u in R, u -> w residual, w in Q, d(w) <= L_k(Q) }).
// For each (region, neighbour) face the pairs (m(u), d(u)), m(u) the least
// finite label u reaches across the face, are reduced to their Pareto
// staircase (m ascending, d ascending) once per call, so a level step is a
// short scan; level 1 (all neighbours at threshold 0) is taken while the
// staircases are built.  Only regions next to a region whose threshold changed
// at the previous level are re-examined.  d'(v) for a vertex of R with label
// x > 0 is the first level k with L_k(R) >= x (d_inf if none); every change of
// L(R) is recorded as a breakpoint (L, k).  Inner vertices use the same rule,
// which keeps the labeling valid (d' is monotone in the label inside a region).
//
// A face with more than kStair staircase steps keeps the first kStair - 1 and
// one step (next m, highest d) for the rest: that only adds arcs to the
// auxiliary graph, so the result stays a valid lower bound (counted in the
// merge counter; 0 means the result is exact).  If the breakpoint pool fills
// up, nothing is applied.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>

#include "mf_internal.cuh"

namespace cg = cooperative_groups;

namespace mf {

namespace {

constexpr int kStair = 8;          // staircase steps kept per (region, neighbour) face
constexpr int kPoolPerRegion = 8;  // breakpoint pool entries per region
constexpr int kBuildWarps = 8;     // warps per block of the staircase build

// scratch layout (all offsets in bytes, 16-aligned)
struct BrLayout {
    size_t stair, lb0, lb1, front0, front1, bphead, bp, bpnext, words, total;
    long long pool;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ inline BrLayout br_layout(const Geom &g, int conn) {
    BrLayout L{};
    const size_t nr = (size_t)g.nreg, faces = nr * (size_t)conn;
    L.pool = (long long)nr * kPoolPerRegion + 1024;
    size_t o = 0;
    L.stair = o;  o += align16(faces * kStair * sizeof(int2));
    L.lb0 = o;    o += align16(nr * 4);
    L.lb1 = o;    o += align16(nr * 4);
    L.front0 = o; o += align16(nr * 4);
    L.front1 = o; o += align16(nr * 4);
    L.bphead = o; o += align16(nr * 4);
    L.bp = o;     o += align16((size_t)L.pool * sizeof(int2));
    L.bpnext = o; o += align16((size_t)L.pool * 4);
    L.words = o;  o += 64;
    L.total = o;
    return L;
}

// words[]: level counters (3, triple-buffered), pool head, overflow, merged faces, levels
enum BrWord { kCnt0 = 0, kPoolHead = 3, kOverflow = 4, kMerged = 5, kLevels = 6, kBrWords = 8 };

// Thresholds live in two buffers by level parity: at the start of level k,
// lb[(k-1)&1][x] = L_{k-1}(x) for every region x; level k raises into
// lb[k&1] (after copying the regions that changed at level k-1 forward), so
// one grid barrier per level suffices.  The staircase of a face is kStair
// int2 (m, d) with unused steps m = INT_MAX.
struct BrPtrs {
    int2 *stair;
    int *lb[2], *front[2], *bphead;
    int2 *bp;
    int *bpnext, *words;
    long long pool;
};

inline BrPtrs br_ptrs(const Geom &g, int conn, void *scratch) {
    const BrLayout L = br_layout(g, conn);
    char *b = (char *)scratch;
    BrPtrs P{};
    P.stair = (int2 *)(b + L.stair);
    P.lb[0] = (int *)(b + L.lb0);
    P.lb[1] = (int *)(b + L.lb1);
    P.front[0] = (int *)(b + L.front0);
    P.front[1] = (int *)(b + L.front1);
    P.bphead = (int *)(b + L.bphead);
    P.bp = (int2 *)(b + L.bp);
    P.bpnext = (int *)(b + L.bpnext);
    P.words = (int *)(b + L.words);
    P.pool = L.pool;
    return P;
}

__device__ __forceinline__ int region_at(const Geom &g, int x, int y, int z) {
    return ((z >> g.sz) * g.RY + (y >> g.sy)) * g.RX + (x >> g.sx);
}

// Staircase of the face of region r toward the neighbour region in direction j
// (the region offset equals the stencil offset of arc direction j).  One warp.
template <int CONN>
__device__ void build_face(const Geom &g, const DevState &st, const BrPtrs &P, int r, int j, int *sm, int *sl,
                           int fmax) {
    const int lane = threadIdx.x & 31;
    const int ox = arc_dx(CONN, j), oy = arc_dy(CONN, j), oz = arc_dz(CONN, j);
    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    const int qx = rx + ox, qy = ry + oy, qz = rz + oz;
    int2 *out = &P.stair[((size_t)r * CONN + j) * kStair];
    if (qx < 0 || qx >= g.RX || qy < 0 || qy >= g.RY || qz < 0 || qz >= g.RZ) {
        if (lane < kStair) out[lane] = make_int2(INT_MAX, 0);
        return;
    }
    const int x0 = rx * g.tx, y0 = ry * g.ty, z0 = rz * g.tz;
    const int ex = min(g.tx, g.X - x0), ey = min(g.ty, g.Y - y0), ez = min(g.tz, g.Z - z0);
    // the face: fixed coordinate on the axes the offset crosses, full range on the others
    const int nx = ox ? 1 : ex, ny = oy ? 1 : ey, nz = oz ? 1 : ez;
    const int fx = ox > 0 ? g.tx - 1 : 0, fy = oy > 0 ? g.ty - 1 : 0, fz = oz > 0 ? g.tz - 1 : 0;
    const int F = nx * ny * nz;  // <= fmax
    const size_t n = (size_t)g.n;
    int lmax_all = 0;
    for (int i = lane; i < F; i += 32) {
        const int lx = ox ? fx : i % nx, ly = oy ? fy : (i / nx) % ny, lz = oz ? fz : i / (nx * ny);
        const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
        const size_t u = ((size_t)z * g.Y + y) * g.X + x;
        const int l = st.lab[u];
        int m = INT_MAX;
        if (l > 0 && l < g.dinf) {
#pragma unroll
            for (int d = 0; d < CONN; ++d) {
                const int dx = arc_dx(CONN, d), dy = arc_dy(CONN, d), dz = arc_dz(CONN, d);
                // only arcs that cross the face's axes in its direction can land in the neighbour
                if ((ox && dx != ox) || (oy && dy != oy) || (oz && dz != oz)) continue;
                const int wx = x + dx, wy = y + dy, wz = z + dz;
                if (wx < 0 || wx >= g.X || wy < 0 || wy >= g.Y || wz < 0 || wz >= g.Z) continue;
                if (region_at(g, wx, wy, wz) != (qz * g.RY + qy) * g.RX + qx) continue;
                if (st.cap[(size_t)d * n + u] <= 0) continue;
                const int lw = st.lab[((size_t)wz * g.Y + wy) * g.X + wx];
                if (lw < g.dinf) m = min(m, lw);
            }
        }
        sm[i] = m;
        sl[i] = l;
        if (m != INT_MAX) lmax_all = max(lmax_all, l);
    }
    __syncwarp();
    lmax_all = __reduce_max_sync(0xffffffffu, lmax_all);
    int k = 0, best = 0, prev = -1, first_m = INT_MAX, first_l = 0;
    bool merged = false;
    while (best < lmax_all && k < kStair) {
        // next distinct reach label above prev, and the highest label reaching it
        int mc = INT_MAX;
        for (int i = lane; i < F; i += 32)
            if (sm[i] != INT_MAX && sm[i] > prev) mc = min(mc, sm[i]);
        mc = (int)__reduce_min_sync(0xffffffffu, (unsigned)mc);
        if (mc == INT_MAX) break;
        int lc = 0;
        for (int i = lane; i < F; i += 32)
            if (sm[i] <= mc) lc = max(lc, sl[i]);
        lc = __reduce_max_sync(0xffffffffu, lc);
        if (lc > best) {
            if (k == kStair - 1 && lc < lmax_all) {  // out of steps: one step for the rest
                lc = lmax_all;
                merged = true;
            }
            if (lane == 0) out[k] = make_int2(mc, lc);
            if (k == 0) {
                first_m = mc;
                first_l = lc;
            }
            ++k;
            best = lc;
        }
        prev = mc;
    }
    if (lane >= k && lane < kStair) out[lane] = make_int2(INT_MAX, 0);
    if (lane == 0) {
        if (merged) atomicAdd(&P.words[kMerged], 1);
        // level 1: the neighbour's threshold L_0 is 0, so the face raises r to
        // the label of its first step if that step reaches label 0
        if (first_m == 0 && first_l > 0) {
            const int old = atomicMax(&P.lb[1][r], first_l);
            if (old == 0) P.front[1][atomicAdd(&P.words[kCnt0 + 1], 1)] = r;
        }
    }
}

template <int CONN>
__global__ void br_build_kernel(const Geom g, const DevState st, const BrPtrs P, int fmax) {
    extern __shared__ int smem[];
    const int w = threadIdx.x >> 5;
    int *sm = smem + (size_t)w * 2 * fmax;
    int *sl = sm + fmax;
    const long long item = (long long)blockIdx.x * kBuildWarps + w;
    if (item >= (long long)g.nreg * CONN) return;
    build_face<CONN>(g, st, P, (int)(item / CONN), (int)(item % CONN), sm, sl, fmax);
}

// Levels 2, 3, ... in one cooperative launch (level 1 is done by the build).
// Level k walks the faces toward every region q raised at level k-1: q's
// threshold is first copied forward into lb[k&1] and its breakpoint
// (L_{k-1}(q), k-1) recorded; then each neighbour r reads its face toward q
// with L_{k-1}(q) and raises lb[k&1][r].  The counters of raised regions are
// triple-buffered so that none is reset while a thread may still read it.
template <int CONN>
__global__ void br_levels_kernel(const Geom g, const BrPtrs P, int max_levels) {
    cg::grid_group grid = cg::this_grid();
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    int *words = P.words;
    int k = 2;
    for (; k <= max_levels; ++k) {
        const bool odd = k & 1;
        const int *fin = odd ? P.front[0] : P.front[1];
        int *fout = odd ? P.front[1] : P.front[0];
        const int *lprev = odd ? P.lb[0] : P.lb[1];
        int *lnew = odd ? P.lb[1] : P.lb[0];
        const int nin = *(volatile int *)&words[kCnt0 + (k - 1) % 3];
        int *cout = &words[kCnt0 + k % 3];
        for (long long t = tid; t < (long long)nin * CONN; t += nth) {
            const int idx = (int)(t / CONN), j = (int)(t % CONN);
            const int q = fin[idx];
            const int Lq = lprev[q];
            if (j == 0) {
                atomicMax(&lnew[q], Lq);
                const int e = atomicAdd(&words[kPoolHead], 1);
                if (e < P.pool) {
                    P.bp[e] = make_int2(Lq, k - 1);
                    P.bpnext[e] = P.bphead[q];
                    P.bphead[q] = e;
                } else {
                    words[kOverflow] = 1;
                }
            }
            const int qx = q % g.RX, qy = (q / g.RX) % g.RY, qz = q / (g.RX * g.RY);
            const int rx = qx + arc_dx(CONN, j), ry = qy + arc_dy(CONN, j), rz = qz + arc_dz(CONN, j);
            if (rx < 0 || rx >= g.RX || ry < 0 || ry >= g.RY || rz < 0 || rz >= g.RZ) continue;
            const int r = (rz * g.RY + ry) * g.RX + rx;
            const int4 *st4 = (const int4 *)&P.stair[((size_t)r * CONN + (j ^ 1)) * kStair];  // r's face toward q
            int4 s4[kStair / 2];
#pragma unroll
            for (int e = 0; e < kStair / 2; ++e) s4[e] = st4[e];
            const int Lr = lprev[r];
            int c = 0;
#pragma unroll
            for (int e = 0; e < kStair / 2; ++e) {
                if (s4[e].x <= Lq) c = s4[e].y;
                if (s4[e].z <= Lq) c = s4[e].w;
            }
            if (c > Lr) {
                const int old = atomicMax(&lnew[r], c);
                if (old <= Lr) fout[atomicAdd(cout, 1)] = r;  // first raise of r at this level
            }
        }
        if (tid == 0) words[kCnt0 + (k + 1) % 3] = 0;
        grid.sync();
        if (*(volatile int *)cout == 0) break;
    }
    if (tid == 0) {
        words[kLevels] = k;
        if (k > max_levels) words[kOverflow] = 1;
    }
}

// d := max(d, d') on every vertex, one block per region: the region's
// breakpoints (newest first: L and level descending) are read into shared
// memory; the boundary-label histogram gets the changes (warp-aggregated);
// the region's activity (an excess vertex below d_inf) is set from the new
// labels and counted.  With an overflowed breakpoint pool the labels stay.
constexpr int kApplyThreads = 256;
constexpr int kBpShared = 64;

__device__ __forceinline__ void hist_move(int *hist, int from, int to, bool on) {
    // every lane of the warp calls this; lanes with on move one count from -> to
    const unsigned act = __ballot_sync(0xffffffffu, on);
    if (!act) return;
    const int lane = threadIdx.x & 31;
    if (on) {
        const unsigned mf = __match_any_sync(act, from);
        if (lane == __ffs(mf) - 1 && from < 0x7fffffff) atomicSub(&hist[from < kHistBins ? from : kHistBins], __popc(mf));
        const unsigned mt = __match_any_sync(act, to);
        if (lane == __ffs(mt) - 1 && to < 0x7fffffff) atomicAdd(&hist[to < kHistBins ? to : kHistBins], __popc(mt));
    }
}

template <int CONN>
__global__ void __launch_bounds__(kApplyThreads) br_apply_kernel(const Geom g, const DevState st, const BrPtrs P) {
    __shared__ int2 sbp[kBpShared];
    __shared__ int s_nbp, s_act;
    const bool apply = P.words[kOverflow] == 0;
    const int V = g.tx * g.ty * g.tz;
    for (int r = blockIdx.x; r < g.nreg; r += gridDim.x) {
        if (threadIdx.x == 0) {
            int nb = 0;
            for (int e = apply ? P.bphead[r] : -1; e >= 0 && nb < kBpShared; e = P.bpnext[e]) sbp[nb++] = P.bp[e];
            s_nbp = nb;
            s_act = 0;
        }
        __syncthreads();
        const int nbp = s_nbp;
        const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
        int act = 0;
        for (int i0 = 0; i0 < V; i0 += kApplyThreads) {
            const int i = i0 + threadIdx.x;
            const int lx = i & (g.tx - 1), ly = (i >> g.sx) & (g.ty - 1), lz = i >> (g.sx + g.sy);
            const int x = rx * g.tx + lx, y = ry * g.ty + ly, z = rz * g.tz + lz;
            const bool in = i < V && x < g.X && y < g.Y && z < g.Z;
            const size_t v = in ? ((size_t)z * g.Y + y) * g.X + x : 0;
            int l = in ? st.lab[v] : 0, nl = l;
            if (in && apply && l > 0 && l < g.dinf) {
                int k = INT_MAX;
                int e = 0;
                for (; e < nbp && sbp[e].x >= l; ++e) k = sbp[e].y;
                if (e == kBpShared) {  // a longer list: walk on in global memory
                    int q = P.bphead[r];
                    for (int s2 = 0; s2 < kBpShared; ++s2) q = P.bpnext[q];
                    for (long long steps = 0; q >= 0 && steps < P.pool; q = P.bpnext[q], ++steps) {
                        const int2 b = P.bp[q];
                        if (b.x < l) break;
                        k = b.y;
                    }
                }
                nl = k == INT_MAX ? g.dinf : min(g.dinf, max(l, k));
                if (nl != l) st.lab[v] = nl;
            }
            const bool border = lx == 0 || lx == g.tx - 1 || ly == 0 || ly == g.ty - 1 ||
                                (CONN == 6 && (lz == 0 || lz == g.tz - 1));
            // in B iff a straight neighbour lies in another region (a diagonal
            // neighbour in another region implies a straight one)
            const bool inB = in && border &&
                             ((lx == 0 && x > 0) || (lx == g.tx - 1 && x + 1 < g.X) || (ly == 0 && y > 0) ||
                              (ly == g.ty - 1 && y + 1 < g.Y) ||
                              (CONN == 6 && ((lz == 0 && z > 0) || (lz == g.tz - 1 && z + 1 < g.Z))));
            hist_move(st.hist, l < g.dinf ? l : 0x7fffffff, nl < g.dinf ? nl : 0x7fffffff, inB && nl != l);
            if (in && nl < g.dinf && !act && st.exc[v] > 0) act = 1;
        }
        act = __syncthreads_or(act);
        if (threadIdx.x == 0) {
            st.active[r] = (unsigned char)act;
            if (act) atomicAdd(&st.ctr[kActiveRegions], 1);
        }
        __syncthreads();
    }
}

int max_face(const Geom &g, int conn) {
    if (conn == 6) return std::max(g.ty * g.tz, std::max(g.tx * g.tz, g.tx * g.ty));
    return std::max(g.tx, g.ty);
}

template <int CONN>
cudaError_t br_impl(const Geom &g, const DevState &st, void *scratch, int *h_words, BrResult *res, cudaStream_t s) {
    const BrPtrs P = br_ptrs(g, CONN, scratch);
    const BrLayout L = br_layout(g, CONN);
    const size_t nr = (size_t)g.nreg;
    cudaError_t e = cudaMemsetAsync((char *)scratch + L.lb0, 0, L.front0 - L.lb0, s);  // both threshold buffers
    if (e == cudaSuccess) e = cudaMemsetAsync(P.bphead, 0xff, nr * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.words, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st.ctr[kActiveRegions], 0, 4, s);
    if (e != cudaSuccess) return e;
    const int fmax = max_face(g, CONN);
    const long long faces = (long long)nr * CONN;
    const size_t smem = (size_t)kBuildWarps * 2 * fmax * 4;
    br_build_kernel<CONN><<<(unsigned)((faces + kBuildWarps - 1) / kBuildWarps), 32 * kBuildWarps, smem, s>>>(
        g, st, P, fmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int max_blocks = 0;
    {
        const cudaError_t e_mb = coop_max_blocks((const void *)br_levels_kernel<CONN>, 256, 0, &max_blocks);
        if (e_mb != cudaSuccess) return e_mb;
    }
    // the level steps are short: a few hundred blocks keep the grid barrier cheap
    const int nblocks = (int)std::max<long long>(1, std::min<long long>({(faces + 255) / 256, (long long)max_blocks, 4ll * device_sms()}));
    Geom gg = g;
    BrPtrs pp = P;
    int max_levels = g.dinf + 1;
    void *args[] = {&gg, &pp, &max_levels};
    e = cudaLaunchCooperativeKernel((const void *)br_levels_kernel<CONN>, dim3(nblocks), dim3(256), args, 0, s);
    if (e != cudaSuccess) return e;
    br_apply_kernel<CONN><<<(unsigned)std::min<size_t>(nr, device_sms() * 16), kApplyThreads, 0, s>>>(g, st, P);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_words, P.words, kBrWords * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    res->levels = h_words[kLevels];
    res->merged = h_words[kMerged];
    res->applied = h_words[kOverflow] == 0;
    res->launches = 3;
    return cudaSuccess;
}

}  // namespace

size_t br_scratch_bytes(const Geom &g, int conn) { return br_layout(g, conn).total; }

cudaError_t boundary_relabel(int conn, const Geom &g, const DevState &st, void *scratch, int *h_words,
                             BrResult *res, cudaStream_t s) {
    if (conn == 4) return br_impl<4>(g, st, scratch, h_words, res, s);
    if (conn == 8) return br_impl<8>(g, st, scratch, h_words, res, s);
    if (conn == 6) return br_impl<6>(g, st, scratch, h_words, res, s);
    return cudaErrorInvalidValue;
}

}  // namespace mf
