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
// short scan.  Only regions next to a region whose threshold changed at the
// previous level are re-examined.  d'(v) for a vertex of R with label x > 0 is
// the first level k with L_k(R) >= x (d_inf if none); every change of L(R) is
// recorded as a breakpoint (L, k).  Inner vertices use the same rule, which
// keeps the labeling valid (d' is monotone in the label inside a region).
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
    size_t stair, scount, lcur, lnext, front0, front1, bphead, bp, bpnext, words, total;
    long long pool;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ inline BrLayout br_layout(const Geom &g, int conn) {
    BrLayout L{};
    const size_t nr = (size_t)g.nreg, faces = nr * (size_t)conn;
    L.pool = (long long)nr * kPoolPerRegion + 1024;
    size_t o = 0;
    L.stair = o;  o += align16(faces * kStair * sizeof(int2));
    L.scount = o; o += align16(faces * 4);
    L.lcur = o;   o += align16(nr * 4);
    L.lnext = o;  o += align16(nr * 4);
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

struct BrPtrs {
    int2 *stair;
    int *scount, *lcur, *lnext, *front0, *front1, *bphead;
    int2 *bp;
    int *bpnext, *words;
    long long pool;
};

inline BrPtrs br_ptrs(const Geom &g, int conn, void *scratch) {
    const BrLayout L = br_layout(g, conn);
    char *b = (char *)scratch;
    return BrPtrs{(int2 *)(b + L.stair), (int *)(b + L.scount), (int *)(b + L.lcur), (int *)(b + L.lnext),
                  (int *)(b + L.front0), (int *)(b + L.front1), (int *)(b + L.bphead), (int2 *)(b + L.bp),
                  (int *)(b + L.bpnext), (int *)(b + L.words), L.pool};
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
    int *cnt = &P.scount[(size_t)r * CONN + j];
    if (qx < 0 || qx >= g.RX || qy < 0 || qy >= g.RY || qz < 0 || qz >= g.RZ) {
        if (lane == 0) *cnt = 0;
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
    int2 *out = &P.stair[((size_t)r * CONN + j) * kStair];
    int k = 0, best = 0, prev = -1;
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
            ++k;
            best = lc;
        }
        prev = mc;
    }
    if (lane == 0) {
        *cnt = k;
        if (merged) atomicAdd(&P.words[kMerged], 1);
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

// All levels in one cooperative launch.  Level k: (A) every face of a region
// next to a region whose threshold changed at level k-1 (all regions at
// k = 1) is read with that neighbour's threshold and raises the region's next
// threshold; (B) the raised regions commit their thresholds and record the
// breakpoint (L, k).  The counters are triple-buffered so that none is reset
// while another thread may still read it.
template <int CONN>
__global__ void br_levels_kernel(const Geom g, const BrPtrs P, int max_levels) {
    cg::grid_group grid = cg::this_grid();
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    int *words = P.words;
    int k = 1;
    for (; k <= max_levels; ++k) {
        const int *fin = (k & 1) ? P.front1 : P.front0;
        int *fout = (k & 1) ? P.front0 : P.front1;
        const int nin = k == 1 ? g.nreg : *(volatile int *)&words[kCnt0 + (k - 1) % 3];
        int *cout = &words[kCnt0 + k % 3];
        for (long long t = tid; t < (long long)nin * CONN; t += nth) {
            const int idx = (int)(t / CONN), j = (int)(t % CONN);
            const int q = k == 1 ? idx : fin[idx];
            const int qx = q % g.RX, qy = (q / g.RX) % g.RY, qz = q / (g.RX * g.RY);
            const int rx = qx + arc_dx(CONN, j), ry = qy + arc_dy(CONN, j), rz = qz + arc_dz(CONN, j);
            if (rx < 0 || rx >= g.RX || ry < 0 || ry >= g.RY || rz < 0 || rz >= g.RZ) continue;
            const int r = (rz * g.RY + ry) * g.RX + rx;
            const size_t f = (size_t)r * CONN + (j ^ 1);  // r's face toward q
            const int Lq = P.lcur[q], Lr = P.lcur[r];
            const int ns = P.scount[f];
            int c = 0;
            for (int e = 0; e < ns; ++e) {
                const int2 s = P.stair[f * kStair + e];
                if (s.x > Lq) break;
                c = s.y;
            }
            if (c > Lr) {
                const int old = atomicMax(&P.lnext[r], c);
                if (old == Lr) fout[atomicAdd(cout, 1)] = r;  // first raise of r at this level
            }
        }
        grid.sync();
        const int nout = *(volatile int *)cout;
        for (long long t = tid; t < nout; t += nth) {
            const int r = fout[t];
            const int L = P.lnext[r];
            P.lcur[r] = L;
            const int e = atomicAdd(&words[kPoolHead], 1);
            if (e < P.pool) {
                P.bp[e] = make_int2(L, k);
                P.bpnext[e] = P.bphead[r];
                P.bphead[r] = e;
            } else {
                words[kOverflow] = 1;
            }
        }
        if (tid == 0) words[kCnt0 + (k + 1) % 3] = 0;
        grid.sync();
        if (nout == 0) break;
    }
    if (tid == 0) {
        words[kLevels] = k;
        if (k > max_levels) words[kOverflow] = 1;
    }
}

// d := max(d, d') on every vertex; rebuild the boundary-label histogram and
// the region activity from the new labels.
template <int CONN>
__global__ void br_apply_kernel(const Geom g, const DevState st, const BrPtrs P) {
    constexpr int SB = 2048;  // labels below SB are counted in shared memory first
    __shared__ int sh[SB];
    for (int b = threadIdx.x; b < SB; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const long long pool = P.pool;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < g.n;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % g.X), y = (int)((v / g.X) % g.Y), z = (int)(v / ((long long)g.X * g.Y));
        const int r = region_at(g, x, y, z);
        int l = st.lab[v];
        if (l > 0 && l < g.dinf) {
            int k = INT_MAX;
            long long steps = 0;
            for (int e = P.bphead[r]; e >= 0 && steps < pool; e = P.bpnext[e], ++steps) {
                const int2 b = P.bp[e];
                if (b.x < l) break;
                k = b.y;
            }
            const int nl = k == INT_MAX ? g.dinf : min(g.dinf, max(l, k));
            if (nl != l) {
                st.lab[v] = nl;
                l = nl;
            }
        }
        if (l >= g.dinf) continue;
        if (st.exc[v] > 0) st.active[r] = 1;
        const int lx = x & (g.tx - 1), ly = y & (g.ty - 1), lz = z & (g.tz - 1);
        const bool border = lx == 0 || lx == g.tx - 1 || ly == 0 || ly == g.ty - 1 ||
                            (CONN == 6 && (lz == 0 || lz == g.tz - 1));
        if (!border) continue;
        bool inB = false;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d), wz = z + arc_dz(CONN, d);
            if (wx < 0 || wx >= g.X || wy < 0 || wy >= g.Y || wz < 0 || wz >= g.Z) continue;
            if (region_at(g, wx, wy, wz) != r) inB = true;
        }
        if (!inB) continue;
        if (l < SB) atomicAdd(&sh[l], 1);
        else atomicAdd(&st.hist[l < kHistBins ? l : kHistBins], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < SB; b += blockDim.x)
        if (sh[b]) atomicAdd(&st.hist[b], sh[b]);
}

__global__ void br_count_active_kernel(const DevState st, int nreg) {
    int c = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreg; r += gridDim.x * blockDim.x) c += st.active[r] != 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st.ctr[kActiveRegions], c);
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
    cudaError_t e = cudaMemsetAsync((char *)scratch + L.lcur, 0, 2 * align16(nr * 4), s);  // lcur, lnext
    if (e == cudaSuccess) e = cudaMemsetAsync(P.bphead, 0xff, nr * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.words, 0, 64, s);
    if (e != cudaSuccess) return e;
    const int fmax = max_face(g, CONN);
    const long long faces = (long long)nr * CONN;
    const size_t smem = (size_t)kBuildWarps * 2 * fmax * 4;
    br_build_kernel<CONN><<<(unsigned)((faces + kBuildWarps - 1) / kBuildWarps), 32 * kBuildWarps, smem, s>>>(
        g, st, P, fmax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static int max_blocks = 0;
    if (!max_blocks) {
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, br_levels_kernel<CONN>, 256, 0);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        max_blocks = per_sm * sms;
        if (max_blocks <= 0) return cudaErrorCooperativeLaunchTooLarge;
    }
    const int nblocks = (int)std::max<long long>(1, std::min<long long>((faces + 255) / 256, max_blocks));
    Geom gg = g;
    BrPtrs pp = P;
    int max_levels = g.dinf + 1;
    void *args[] = {&gg, &pp, &max_levels};
    e = cudaLaunchCooperativeKernel((const void *)br_levels_kernel<CONN>, dim3(nblocks), dim3(256), args, 0, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_words, P.words, kBrWords * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    res->levels = h_words[kLevels];
    res->merged = h_words[kMerged];
    res->applied = h_words[kOverflow] == 0;
    res->launches = 2;
    if (!res->applied) return cudaSuccess;
    e = cudaMemsetAsync(st.hist, 0, (kHistBins + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st.active, 0, nr, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&st.ctr[kActiveRegions], 0, 4, s);
    if (e != cudaSuccess) return e;
    const int nb = (int)std::min<long long>((g.n + 255) / 256, 152 * 32);
    br_apply_kernel<CONN><<<nb, 256, 0, s>>>(g, st, P);
    br_count_active_kernel<<<(g.nreg + 255) / 256, 256, 0, s>>>(st, g.nreg);
    res->launches += 2;
    return cudaGetLastError();
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
