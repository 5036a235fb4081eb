// Region reduction (Sec. 8, the Region Reduction algorithm): a preprocessing
// that decides vertices from one region's network alone.
//
// For every region R of a tiling, one thread block holds the region network
// G^R in shared memory: the vertices of R with their terminal links, the
// boundary B^R (the vertices outside R adjacent to R, without terminal links
// and without arcs among themselves), the arcs inside R and the arcs between
// R and B^R in both directions.  It is laid out as the tile plus a one-cell
// ring (the ring cells that are adjacent to R form B^R).  The block runs the
// section's steps on a preflow (every s-link saturated at the start, so "s
// reaches v" is "v lies in the residual closure of the excess vertices"):
//   1. Augment(s, t): rounds of "exact BFS to the sinks, then a layered push
//      from the highest layer down" until no excess vertex reaches t;
//   2. B^S = boundary vertices reachable from s, B^T = boundary vertices
//      that reach t;
//   3. Augment(s, B^S): the same rounds with every B^S vertex an absorbing
//      sink (an infinite arc into a super sink that is removed afterwards);
//   4. Augment(B^T, t): every B^T vertex gets a supply equal to its residual
//      out-capacity (no flow out of it can exceed that, so the supply acts as
//      an infinite arc from a super source), the same rounds; the supply that
//      got stuck on the way is pushed back to B^T (so that the residual
//      network is that of a maximum flow from B^T to t, not of a preflow), and
//      what is left at B^T is dropped with the super source;
//   5. classes of the vertices of R in the final residual network: s -> v
//      strong source, v -> t strong sink, otherwise weak source if v does not
//      reach B^R and weak sink if B^R does not reach v.
// Every set the classes are read from is a residual closure computed to its
// fixed point; the pushes follow the same safety rules as the discharge
// kernels (from an excess vertex, along a residual arc, one BFS layer down).
#include <algorithm>
#include <climits>
#include <cstdint>

#include "mf_internal.cuh"

namespace mf {

namespace {

constexpr int kRedThreads = 256;
constexpr int kDistInf = 0x3fffffff;

// per-cell flags (fl) and closure bits (cl)
constexpr unsigned char F_R = 1, F_B = 2, F_BS = 4, F_BT = 8;
constexpr unsigned char C_S = 1, C_T = 2, C_TOB = 4, C_FROMB = 8;

template <int CONN>
__device__ __forceinline__ int cell_off(const RedGeom &rg, int d) {
    return arc_dx(CONN, d) + arc_dy(CONN, d) * rg.EX + arc_dz(CONN, d) * rg.EX * rg.EY;
}

template <int CONN>
__global__ void __launch_bounds__(kRedThreads) region_reduction_kernel(const RedGeom rg, const int *__restrict__ cs,
                                                                       const int *__restrict__ ct,
                                                                       const int *__restrict__ nl,
                                                                       unsigned char *codes,
                                                                       unsigned long long *counts, int max_rounds,
                                                                       int *err) {
    constexpr int N = CONN;
    const int E = rg.E;
    extern __shared__ __align__(16) int sm[];
    int *cap = sm;                 // [N][E] residual capacity of the arc c -> c + D(d) in G^R
    int *tcap = cap + N * E;       // [E] residual of c -> t
    int *exc = tcap + E;           // [E] excess
    int *dist = exc + E;           // [E] BFS layer (1 = next to a sink)
    unsigned char *am = (unsigned char *)(dist + E);  // [E] arcs of G^R leaving the cell (bit d)
    unsigned char *fl = am + E;    // [E] F_* flags
    unsigned char *cl = fl + E;    // [E] closure bits
    __shared__ int s_max;
    __shared__ unsigned long long s_cnt[4];

    const int tid = threadIdx.x;
    const int r = blockIdx.x;
    const int rxi = r % rg.RX, ryi = (r / rg.RX) % rg.RY, rzi = r / (rg.RX * rg.RY);
    const int ox = rxi * rg.tx - 1, oy = ryi * rg.ty - 1, oz = CONN == 6 ? rzi * rg.tz - 1 : 0;
    const size_t n = (size_t)rg.X * rg.Y * rg.Z;
    if (tid < 4) s_cnt[tid] = 0;

    auto cell_xyz = [&](int c, int &ex, int &ey, int &ez) {
        ex = c % rg.EX;
        ey = (c / rg.EX) % rg.EY;
        ez = c / (rg.EX * rg.EY);
    };
    auto in_grid = [&](int x, int y, int z) { return x >= 0 && x < rg.X && y >= 0 && y < rg.Y && z >= 0 && z < rg.Z; };
    auto in_r = [&](int ex, int ey, int ez) {
        const bool zin = CONN != 6 || (ez >= 1 && ez <= rg.tz);
        return ex >= 1 && ex <= rg.tx && ey >= 1 && ey <= rg.ty && zin && in_grid(ox + ex, oy + ey, oz + ez);
    };
    auto in_e = [&](int ex, int ey, int ez) { return ex >= 0 && ex < rg.EX && ey >= 0 && ey < rg.EY && ez >= 0 && ez < rg.EZ; };

    // ---- the region network -------------------------------------------------------
    for (int c = tid; c < E; c += kRedThreads) {
        int ex, ey, ez;
        cell_xyz(c, ex, ey, ez);
        const int x = ox + ex, y = oy + ey, z = oz + ez;
        const bool gin = in_grid(x, y, z);
        const bool rin = in_r(ex, ey, ez);
        const size_t v = gin ? ((size_t)z * rg.Y + y) * rg.X + x : 0;
        unsigned char amask = 0, f = rin ? F_R : 0;
#pragma unroll
        for (int d = 0; d < N; ++d) {
            const int wx = ex + arc_dx(CONN, d), wy = ey + arc_dy(CONN, d), wz = ez + arc_dz(CONN, d);
            int c_arc = 0;
            if (gin && in_e(wx, wy, wz) && in_grid(ox + wx, oy + wy, oz + wz)) {
                const bool win = in_r(wx, wy, wz);
                if (rin || win) {  // arcs of G^R: inside R, or between R and B^R
                    const int h = d >> 1;
                    const size_t w = ((size_t)(oz + wz) * rg.Y + (oy + wy)) * rg.X + (ox + wx);
                    c_arc = (d & 1) ? nl[(size_t)h * n + w] : nl[(size_t)h * n + v];
                    amask |= (unsigned char)(1u << d);
                    if (!rin) f |= F_B;  // a cell outside R with an arc into R belongs to B^R
                }
            }
            cap[d * E + c] = c_arc;
        }
        int e = 0, tc = 0;
        if (rin) {
            const int a = cs[v], b = ct[v];
            const int m = min(a, b);  // sent s -> v -> t at once
            e = a - m;
            tc = b - m;
        }
        exc[c] = e;
        tcap[c] = tc;
        am[c] = amask;
        fl[c] = f;
        cl[c] = 0;
    }
    __syncthreads();

    // ---- Augment: rounds of BFS to the sinks + layered push ------------------------
    // sinks: a residual arc to t (use_t), and the vertices flagged `absorb`
    // (each with an infinite arc into a super sink)
    auto bfs = [&](unsigned char absorb, bool use_t) -> int {
        for (int c = tid; c < E; c += kRedThreads)
            dist[c] = ((use_t && tcap[c] > 0) || (fl[c] & absorb)) ? 1 : kDistInf;
        if (tid == 0) s_max = 0;
        __syncthreads();
        for (int L = 1;; ++L) {
            int changed = 0;
            for (int c = tid; c < E; c += kRedThreads) {
                if (dist[c] != kDistInf) continue;
                const unsigned a = am[c];
#pragma unroll
                for (int d = 0; d < N; ++d) {
                    if (!((a >> d) & 1u) || cap[d * E + c] <= 0) continue;
                    if (dist[c + cell_off<CONN>(rg, d)] == L) {
                        dist[c] = L + 1;
                        changed = 1;
                        break;
                    }
                }
            }
            if (!__syncthreads_or(changed)) break;
        }
        int lm = 0;
        for (int c = tid; c < E; c += kRedThreads)
            if (exc[c] > 0 && dist[c] != kDistInf) lm = max(lm, dist[c]);
        if (lm) atomicMax(&s_max, lm);
        __syncthreads();
        const int res = s_max;
        __syncthreads();
        return res;
    };
    auto push = [&](int Lmax, unsigned char absorb, bool use_t) {
        for (int L = Lmax; L >= 1; --L) {
            for (int c = tid; c < E; c += kRedThreads) {
                if (dist[c] != L) continue;
                int e = exc[c];
                if (e <= 0) continue;
                if (L == 1) {
                    const int tc = use_t ? tcap[c] : 0;
                    if (tc > 0) {
                        const int dl = min(e, tc);
                        tcap[c] = tc - dl;
                        e -= dl;
                    }
                    if (fl[c] & absorb) e = 0;  // into the super sink
                } else {
                    const unsigned a = am[c];
#pragma unroll
                    for (int d = 0; d < N; ++d) {
                        if (e == 0) break;
                        if (!((a >> d) & 1u)) continue;
                        const int cc = cap[d * E + c];
                        if (cc <= 0) continue;
                        const int w = c + cell_off<CONN>(rg, d);
                        if (dist[w] != L - 1) continue;
                        const int dl = min(e, cc);
                        cap[d * E + c] = cc - dl;
                        cap[(d ^ 1) * E + w] += dl;
                        atomicAdd(&exc[w], dl);
                        e -= dl;
                    }
                }
                exc[c] = e;
            }
            __syncthreads();
        }
    };
    bool ok = true;
    auto augment = [&](unsigned char absorb, bool use_t) {
        for (int round = 0; ok; ++round) {
            if (round >= max_rounds) {
                ok = false;
                break;
            }
            const int Lmax = bfs(absorb, use_t);
            if (Lmax == 0) break;
            push(Lmax, absorb, use_t);
        }
    };
    // residual closure of the cells with bit `bit` set in cl (seeded by the
    // caller): forward = cells reachable from the set, backward = cells that
    // reach the set
    auto closure = [&](unsigned char bit, bool forward) {
        for (;;) {
            int changed = 0;
            for (int c = tid; c < E; c += kRedThreads) {
                if (cl[c] & bit) continue;
                const unsigned a = am[c];
                bool join = false;
#pragma unroll
                for (int d = 0; d < N && !join; ++d) {
                    if (!((a >> d) & 1u)) continue;  // G^R arcs are symmetric: c -> w exists iff w -> c does
                    const int w = c + cell_off<CONN>(rg, d);
                    if (!(cl[w] & bit)) continue;
                    join = forward ? cap[(d ^ 1) * E + w] > 0 : cap[d * E + c] > 0;
                }
                if (join) {
                    cl[c] |= bit;
                    changed = 1;
                }
            }
            if (!__syncthreads_or(changed)) break;
        }
    };

    // 1. Augment(s, t)
    augment(0, true);
    // 2. B^S: boundary vertices in the closure of the excess; B^T: boundary
    //    vertices that reach t
    for (int c = tid; c < E; c += kRedThreads) {
        unsigned char b = 0;
        if (exc[c] > 0) b |= C_S;
        if (tcap[c] > 0) b |= C_T;
        cl[c] = b;
    }
    __syncthreads();
    closure(C_S, true);
    closure(C_T, false);
    for (int c = tid; c < E; c += kRedThreads) {
        if (!(fl[c] & F_B)) continue;
        if (cl[c] & C_S) fl[c] |= F_BS;
        if (cl[c] & C_T) fl[c] |= F_BT;
    }
    __syncthreads();
    // 3. Augment(s, B^S)
    augment(F_BS, true);
    // strong sources: the closure of the excess left (B^S absorbed theirs);
    // step 4 works where s does not reach, so this set stays final
    for (int c = tid; c < E; c += kRedThreads) cl[c] = exc[c] > 0 ? C_S : 0;
    __syncthreads();
    closure(C_S, true);
    // 4. Augment(B^T, t) from a supply at every B^T vertex
    for (int c = tid; c < E; c += kRedThreads) {
        if (!(fl[c] & F_BT)) continue;
        long long sup = exc[c];
        const unsigned a = am[c];
#pragma unroll
        for (int d = 0; d < N; ++d)
            if ((a >> d) & 1u) sup += cap[d * E + c];
        exc[c] = (int)min(sup, (long long)INT_MAX);
    }
    __syncthreads();
    augment(0, true);
    // The supply that did not reach t sits as excess on the way; in a flow
    // (not a preflow) it would never have left B^T, and the arcs it used
    // would still be residual.  Push it back to B^T (B^T absorbing, t not a
    // sink): what is left is a maximum flow from B^T to t.  The excess of the
    // strong sources cannot reach B^R and stays.
    augment(F_BT, false);
    for (int c = tid; c < E; c += kRedThreads)
        if (fl[c] & F_BT) exc[c] = 0;  // the super source leaves with its supply
    // 5. final closures: v -> t, v -> B^R, B^R -> v
    for (int c = tid; c < E; c += kRedThreads) {
        unsigned char b = cl[c] & C_S;
        if (tcap[c] > 0) b |= C_T;
        if (fl[c] & F_B) b |= C_TOB | C_FROMB;
        cl[c] = b;
    }
    __syncthreads();
    closure(C_T, false);
    closure(C_TOB, false);
    closure(C_FROMB, true);

    // ---- classes of the vertices of R --------------------------------------------
    unsigned long long cnt[4] = {0, 0, 0, 0};
    for (int c = tid; c < E; c += kRedThreads) {
        if (!(fl[c] & F_R)) continue;
        int ex, ey, ez;
        cell_xyz(c, ex, ey, ez);
        const size_t v = ((size_t)(oz + ez) * rg.Y + (oy + ey)) * rg.X + (ox + ex);
        const unsigned char b = cl[c];
        unsigned char code = 0;
        if (b & C_S) code |= kStrongSource;
        if (b & C_T) code |= kStrongSink;
        if (!code) {
            if (!(b & C_TOB)) code |= kWeakSource;
            if (!(b & C_FROMB)) code |= kWeakSink;
        }
        codes[v] = code;
        cnt[0] += (code & kStrongSource) != 0;
        cnt[1] += (code & kStrongSink) != 0;
        cnt[2] += (code & kWeakSource) != 0;
        cnt[3] += (code & kWeakSink) != 0;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        unsigned long long x = cnt[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((tid & 31) == 0 && x) atomicAdd(&s_cnt[k], x);
    }
    __syncthreads();
    if (tid < 4 && s_cnt[tid]) atomicAdd(&counts[tid], s_cnt[tid]);
    if (tid == 0 && !ok) atomicExch(err, 1);
}

// Reduced capacities: the strong sources are merged into s and the strong
// sinks into t (every minimum cut already puts them there).  For a vertex w
// left open, cs'(w) = cs(w) + c(edges to strong sources), ct'(w) = ct(w) +
// c(edges to strong sinks), and its edges to decided vertices are removed; a
// decided vertex keeps no link.  The cut edges between the merged sets add
// the constant  sum_{S*} ct + sum_{T*} cs + c(S*, T*)  to every cut (into
// flow0 through *konst).
template <int CONN>
__global__ void reduction_apply_kernel(const Geom g, const unsigned char *__restrict__ codes,
                                       const int *__restrict__ cs, const int *__restrict__ ct,
                                       const int *__restrict__ nl, int *cs2, int *ct2, int *nl2,
                                       unsigned long long *konst, unsigned long long *konst2) {
    const size_t n = (size_t)g.n;
    unsigned long long part = 0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % g.X), y = (int)((v / g.X) % g.Y), z = (int)(v / ((size_t)g.X * g.Y));
        const unsigned char cv = codes[v];
        const bool sv = cv & kStrongSource, tv = cv & kStrongSink;
        long long add_s = 0, add_t = 0;
#pragma unroll
        for (int d = 0; d < CONN; ++d) {
            const int wx = x + arc_dx(CONN, d), wy = y + arc_dy(CONN, d), wz = z + arc_dz(CONN, d);
            if (wx < 0 || wx >= g.X || wy < 0 || wy >= g.Y || wz < 0 || wz >= g.Z) continue;
            const size_t w = ((size_t)wz * g.Y + wy) * g.X + wx;
            const int c = (d & 1) ? nl[(size_t)(d >> 1) * n + w] : nl[(size_t)(d >> 1) * n + v];
            const unsigned char cw = codes[w];
            const bool sw = cw & kStrongSource, tw = cw & kStrongSink;
            if (!(d & 1)) {  // each edge once, at its forward tail
                nl2[(size_t)(d >> 1) * n + v] = (sv || tv || sw || tw) ? 0 : c;
                if ((sv && tw) || (tv && sw)) part += (unsigned long long)c;
            }
            if (!(sv || tv)) {
                if (sw) add_s += c;
                if (tw) add_t += c;
            }
        }
        if (sv || tv) {
            cs2[v] = 0;
            ct2[v] = 0;
            part += (unsigned long long)(sv ? ct[v] : cs[v]);
        } else {
            cs2[v] = (int)(cs[v] + add_s);  // <= cs + all edge capacities at v (checked at set_caps)
            ct2[v] = (int)(ct[v] + add_t);
        }
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part) {
        atomicAdd(konst, part);
        atomicAdd(konst2, part);
    }
}

// S_min |= S*, S_max &= ~T* after the cut of the reduced network
__global__ void reduction_cut_kernel(size_t n, const unsigned char *__restrict__ codes, unsigned char *smin,
                                     unsigned char *smax) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
        const unsigned char c = codes[v];
        if (c & kStrongSource) smin[v] = 1;
        if (c & kStrongSink) smax[v] = 0;
    }
}

}  // namespace

bool reduction_supported(int conn, const int tile[3], RedGeom *out, const Geom &g) {
    const int tx = tile[0], ty = tile[1], tz = conn == 6 ? tile[2] : 1;
    if (tx < 1 || ty < 1 || tz < 1) return false;
    RedGeom rg{};
    rg.X = g.X; rg.Y = g.Y; rg.Z = g.Z;
    rg.tx = tx; rg.ty = ty; rg.tz = tz;
    rg.RX = (g.X + tx - 1) / tx; rg.RY = (g.Y + ty - 1) / ty; rg.RZ = (g.Z + tz - 1) / tz;
    rg.EX = tx + 2; rg.EY = ty + 2; rg.EZ = conn == 6 ? tz + 2 : 1;
    rg.E = rg.EX * rg.EY * rg.EZ;
    if (reduction_smem_bytes(conn, rg) > (size_t)kRedMaxSmem) return false;
    if (out) *out = rg;
    return true;
}

size_t reduction_smem_bytes(int conn, const RedGeom &rg) { return (size_t)rg.E * ((conn + 3) * 4 + 3); }

cudaError_t launch_region_reduction(int conn, const RedGeom &rg, const int *cs, const int *ct, const int *nl,
                                    unsigned char *codes, unsigned long long *counts, int max_rounds, int *err,
                                    cudaStream_t s) {
    const void *k = conn == 4 ? (const void *)region_reduction_kernel<4>
                  : conn == 8 ? (const void *)region_reduction_kernel<8>
                              : (const void *)region_reduction_kernel<6>;
    const size_t smem = reduction_smem_bytes(conn, rg);
    cudaError_t e = ensure_smem_attr(k, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)rg.RX * rg.RY * rg.RZ;
    if (conn == 4) region_reduction_kernel<4><<<blocks, kRedThreads, smem, s>>>(rg, cs, ct, nl, codes, counts, max_rounds, err);
    else if (conn == 8) region_reduction_kernel<8><<<blocks, kRedThreads, smem, s>>>(rg, cs, ct, nl, codes, counts, max_rounds, err);
    else region_reduction_kernel<6><<<blocks, kRedThreads, smem, s>>>(rg, cs, ct, nl, codes, counts, max_rounds, err);
    return cudaGetLastError();
}

cudaError_t launch_reduction_apply(int conn, const Geom &g, const unsigned char *codes, const int *cs, const int *ct,
                                   const int *nl, int *cs2, int *ct2, int *nl2, unsigned long long *konst,
                                   unsigned long long *konst2, cudaStream_t s) {
    const size_t b = ((size_t)g.n + 255) / 256;
    const unsigned blocks = (unsigned)std::min<size_t>(b ? b : 1, (size_t)device_sms() * 16);
    if (conn == 4) reduction_apply_kernel<4><<<blocks, 256, 0, s>>>(g, codes, cs, ct, nl, cs2, ct2, nl2, konst, konst2);
    else if (conn == 8) reduction_apply_kernel<8><<<blocks, 256, 0, s>>>(g, codes, cs, ct, nl, cs2, ct2, nl2, konst, konst2);
    else reduction_apply_kernel<6><<<blocks, 256, 0, s>>>(g, codes, cs, ct, nl, cs2, ct2, nl2, konst, konst2);
    return cudaGetLastError();
}

cudaError_t launch_reduction_cut(size_t n, const unsigned char *codes, unsigned char *smin, unsigned char *smax,
                                 cudaStream_t s) {
    const size_t b = (n + 255) / 256;
    const unsigned blocks = (unsigned)std::min<size_t>(b ? b : 1, (size_t)device_sms() * 16);
    reduction_cut_kernel<<<blocks, 256, 0, s>>>(n, codes, smin, smax);
    return cudaGetLastError();
}

}  // namespace mf
