// Region discharge of P-ARD for 2D tiles with bit-parallel graph search.
//
// Same computation as ard_discharge.cu (Procedure ARD of Sec. 4.2 with
// Procedure Augment done in synchronous rounds of "BFS from T_k, then a
// layered push from the highest BFS layer down", followed by the ARD
// region-relabel of Sec. 5.1), organised for a 64- or 32-wide tile:
//
//   * the residual graph of the tile is also kept as bit masks, one machine
//     word per tile row and arc direction: R_d[y] bit x = [c_f((x,y) -> (x,y)+D(d)) > 0];
//     T[y] bit x = [c_f(v,t) > 0]; E[y] bit x = [e_f(v) > 0];
//   * warp 0 (the "graph warp") runs every BFS and every reachability flood on
//     these masks: lane l holds rows l*RPL .. l*RPL+RPL-1 in registers, a BFS
//     step is a handful of shifts/ands per row plus two warp shuffles for the
//     rows above and below, with no block barrier;
//   * all warps do the per-vertex integer work (tile staging, the layered
//     push, write-back) and keep the masks current with shared-memory atomics.
//
// BFS distances are stored as (epoch << 16 | layer) so no per-round reset of
// the distance array is needed.
#include <climits>
#include <cstdint>

#include "mf_internal.cuh"

namespace mf {

typedef unsigned long long u64;

template <int CONN, int TX, int TY, int NT>
struct Cfg2D {
    static constexpr int N = CONN;
    static constexpr int V = TX * TY;
    static constexpr int NW = NT / 32;                  // warps
    static constexpr int VPT = V / NT;
    static constexpr int RPL = TY / 32;                 // rows per lane of the graph warp
    static constexpr int HL = 2 * (TX + 2) + 2 * TY;    // halo cells (B^R plus unused corners)
    static constexpr int PER = 2 * TX + 2 * (TY - 2);   // perimeter positions of the tile
    static constexpr int LCAP = 64;                     // BFS layers kept as masks
    static constexpr size_t smem = (size_t)(N + 3) * V * 4                  // cap, tcap, exc, lab
                                   + (size_t)(N + 5) * TY * 8               // R[N], T, E, seed, inc, vis
                                   + (size_t)(LCAP + 1) * TY * 8            // BFS layers 1..LCAP
                                   + (size_t)HL * 4 + 64;
    static_assert(TX == 32 || TX == 64, "row width must be 32 or 64");
    static_assert(TY % 32 == 0 && V % NT == 0 && NT % 32 == 0, "tile/threads mismatch");
};

// halo cell index of (hx, hy), a cell just outside the tile
template <int TX, int TY>
__device__ __forceinline__ int halo_idx(int hx, int hy) {
    if (hy < 0) return hx + 1;
    if (hy >= TY) return (TX + 2) + hx + 1;
    if (hx < 0) return 2 * (TX + 2) + hy;
    return 2 * (TX + 2) + TY + hy;
}

// Kogge-Stone fill inside one row: x joins if x+1 is in g and pl[x] (arc x -> x+1),
// or x-1 is in g and pr[x] (arc x -> x-1), repeatedly (a whole run at once).
__device__ __forceinline__ u64 row_fill(u64 g, u64 pl, u64 pr) {
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

// distance tag of a deep BFS layer (negative: never equal to a label >= 0)
__device__ __forceinline__ int deep_tag(int epoch, int L) { return ~((epoch << 16) | L); }

template <int CONN, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, 1)
ard_discharge2d_kernel(const Geom g, const DevState st, const SweepArgs sa) {
    using C = Cfg2D<CONN, TX, TY, NT>;
    constexpr int N = C::N, V = C::V, VPT = C::VPT, RPL = C::RPL, NW = C::NW, LCAP = C::LCAP;
    constexpr int HW = TX / 32;  // 32-bit halves per row
    extern __shared__ __align__(16) unsigned char smraw[];
    int *s_cap = (int *)smraw;            // [N][V] residual of arc i -> i + D(d)
    int *s_tcap = s_cap + N * V;          // [V]
    int *s_exc = s_tcap + V;              // [V]
    int *s_lab = s_exc + V;               // [V] region label (deep BFS layers: negative tags)
    u64 *s_R = (u64 *)(s_lab + V);        // [N][TY] residual masks
    u64 *s_T = s_R + N * TY;              // [TY] residual arc to t
    u64 *s_E = s_T + TY;                  // [TY] positive excess
    u64 *s_seed = s_E + TY;               // [TY] stage seeds (arcs into T_k \ {t})
    u64 *s_inc = s_seed + TY;             // [TY] vertices that joined the closure
    u64 *s_vis = s_inc + TY;              // [TY] final closure
    u64 *s_layer = s_vis + TY;            // [LCAP+1][TY] BFS layers
    int *s_hl = (int *)(s_layer + (LCAP + 1) * TY);  // [HL] labels of B^R
    __shared__ int s_ctl[4];
    __shared__ unsigned long long s_flow;

    const int r = blockIdx.x;
    if (!st.active[r]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rx = r % g.RX, ry = r / g.RX;
    const int ox = rx * TX, oy = ry * TY;
    const size_t n = (size_t)g.n;
    const int dinf = g.dinf;
    if (tid == 0) s_flow = 0;

    // ---- stage the tile; build the masks with warp ballots ---------------------
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        const int i = tid + q * NT;
        const int lx = i % TX, ly = i / TX;
        const int x = ox + lx, y = oy + ly;
        const bool in = x < g.X && y < g.Y;
        const size_t v = (size_t)y * g.X + x;
        int tc = 0, ex = 0;
#pragma unroll
        for (int d = 0; d < N; ++d) {
            const int c = in ? st.cap[d * n + v] : 0;
            s_cap[d * V + i] = c;
            const unsigned b = __ballot_sync(0xffffffffu, c > 0);
            if (lane == 0) ((unsigned *)s_R)[(d * TY + ly) * 2 + (lx >> 5)] = b;
        }
        if (in) {
            tc = st.tcap[v];
            ex = st.exc[v];
        }
        s_tcap[i] = tc;
        s_exc[i] = ex;
        s_lab[i] = 0;
        const unsigned bt = __ballot_sync(0xffffffffu, tc > 0);
        const unsigned be = __ballot_sync(0xffffffffu, ex > 0);
        if (lane == 0) {
            ((unsigned *)s_T)[ly * 2 + (lx >> 5)] = bt;
            ((unsigned *)s_E)[ly * 2 + (lx >> 5)] = be;
        }
    }
    if (TX == 32) {  // upper halves of the row words are never written above
        for (int w = tid; w < (N + 2) * TY; w += NT) ((unsigned *)s_R)[w * 2 + 1] = 0;
    }
    for (int h = tid; h < C::HL; h += NT) {
        int hx, hy;
        if (h < TX + 2) { hx = h - 1; hy = -1; }
        else if (h < 2 * (TX + 2)) { hx = h - (TX + 2) - 1; hy = TY; }
        else if (h < 2 * (TX + 2) + TY) { hx = -1; hy = h - 2 * (TX + 2); }
        else { hx = TX; hy = h - 2 * (TX + 2) - TY; }
        const bool corner = (hx < 0 || hx >= TX) && (hy < 0 || hy >= TY);
        const int x = ox + hx, y = oy + hy;
        const bool ing = x >= 0 && x < g.X && y >= 0 && y < g.Y;
        s_hl[h] = (ing && (CONN == 8 || !corner)) ? st.lab[(size_t)y * g.X + x] : dinf;
    }
    __syncthreads();

    // ---- graph-warp helpers (warp 0) ------------------------------------------
    // next stage value above k: min{d(w)+1 > k : w in B^R, d(w) < d_inf}
    auto next_stage = [&](int k) -> int {
        int best = INT_MAX;
        for (int h = lane; h < C::HL; h += 32) {
            const int v = s_hl[h];
            if (v < dinf && v + 1 > k && v + 1 < best) best = v + 1;
        }
        return __reduce_min_sync(0xffffffffu, best);
    };
    // s_seed[y] bit x = vertex (x,y) has a residual arc to a boundary vertex w with d(w) < k
    auto halo_seeds = [&](int k) {
        for (int y = lane; y < TY; y += 32) s_seed[y] = 0;
        __syncwarp();
        if (k > 0) {
            for (int p = lane; p < C::PER; p += 32) {
                int x, y;
                if (p < TX) { x = p; y = 0; }
                else if (p < 2 * TX) { x = p - TX; y = TY - 1; }
                else if (p < 2 * TX + TY - 2) { x = 0; y = p - 2 * TX + 1; }
                else { x = TX - 1; y = p - (2 * TX + TY - 2) + 1; }
                bool s = false;
#pragma unroll
                for (int d = 0; d < N; ++d) {
                    const int hx = x + arc_dx(CONN, d), hy = y + arc_dy(CONN, d);
                    if (hx >= 0 && hx < TX && hy >= 0 && hy < TY) continue;
                    if (!((s_R[d * TY + y] >> x) & 1ull)) continue;
                    if (s_hl[halo_idx<TX, TY>(hx, hy)] < k) s = true;
                }
                if (s) atomicOr(&s_seed[y], 1ull << x);
            }
        }
        __syncwarp();
    };
    auto load_masks = [&](u64 (&Rm)[N][RPL]) {
#pragma unroll
        for (int j = 0; j < RPL; ++j)
#pragma unroll
            for (int d = 0; d < N; ++d) Rm[d][j] = s_R[d * TY + lane * RPL + j];
    };
    // one backward BFS step on the masks: vertices with a residual arc into f
    auto expand = [&](const u64 (&Rm)[N][RPL], const u64 (&f)[RPL], u64 (&out)[RPL]) {
        const u64 up = __shfl_up_sync(0xffffffffu, f[RPL - 1], 1);
        const u64 dn = __shfl_down_sync(0xffffffffu, f[0], 1);
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const u64 fa = j == 0 ? (lane == 0 ? 0ull : up) : f[j - 1];         // row y-1
            const u64 fb = j == RPL - 1 ? (lane == 31 ? 0ull : dn) : f[j + 1];  // row y+1
            u64 a = (Rm[0][j] & (f[j] >> 1)) | (Rm[1][j] & (f[j] << 1)) | (Rm[2][j] & fb) | (Rm[3][j] & fa);
            if (CONN == 8)
                a |= (Rm[4][j] & (fb >> 1)) | (Rm[5][j] & (fa << 1)) | (Rm[6][j] & (fb << 1)) | (Rm[7][j] & (fa >> 1));
            out[j] = a;
        }
    };
    // closure C := C U {u : u -> seeds of stage k} (reachability, no distances);
    // the vertices that joined go to s_inc; returns whether C meets the excess
    u64 Cl[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) Cl[j] = 0;
    auto closure_extend = [&](int k) -> bool {
        halo_seeds(k);
        u64 Rm[N][RPL], fr[RPL], inc[RPL];
        load_masks(Rm);
        bool any = false;
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int y = lane * RPL + j;
            const u64 sd = (k == 0 ? s_T[y] : s_seed[y]) & ~Cl[j];
            const u64 f = row_fill(sd, Rm[0][j] & ~Cl[j], Rm[1][j] & ~Cl[j]);
            Cl[j] |= f;
            inc[j] = f;
            fr[j] = f;
            any |= f != 0ull;
        }
        while (__any_sync(0xffffffffu, any)) {
            u64 nf[RPL];
            expand(Rm, fr, nf);
            any = false;
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                const u64 f = row_fill(nf[j] & ~Cl[j], Rm[0][j] & ~Cl[j], Rm[1][j] & ~Cl[j]);
                Cl[j] |= f;
                inc[j] |= f;
                fr[j] = f;
                any |= f != 0ull;
            }
        }
        bool meets = false;
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int y = lane * RPL + j;
            s_inc[y] = inc[j];
            meets |= (Cl[j] & s_E[y]) != 0ull;
        }
        return __any_sync(0xffffffffu, meets);
    };
    // all threads: label the vertices that joined the closure at stage k
    auto write_labels = [&](int k) {
        for (int y = warp; y < TY; y += NW) {
            const u64 m = s_inc[y];
            if (!m) continue;
#pragma unroll
            for (int h = 0; h < HW; ++h) {
                const int x = lane + 32 * h;
                if ((m >> x) & 1ull) s_lab[y * TX + x] = k;
            }
        }
    };

    const int klimit = sa.partial ? sa.sweep : INT_MAX;
    long long flow_acc = 0;
    int rounds = 0, stages = 0, epoch = 0;
    bool err = false;

    // ---- ARD stages ------------------------------------------------------------
    for (int k = 0;;) {
        if (warp == 0) {
            const bool reach = closure_extend(k);
            const int kn = next_stage(k);
            if (lane == 0) {
                s_ctl[0] = reach;
                s_ctl[1] = kn;
            }
        }
        __syncthreads();
        write_labels(k);
        const int reach = s_ctl[0], kn = s_ctl[1];
        // after a round-cap error no more augmentation, but the labels of every
        // stage are still computed so the labeling stays valid
        const bool aug = k <= klimit && !err;
        if (aug) ++stages;
        if (aug && reach) {
            // Augment(R, T_k): rounds of exact BFS + layered push
            for (int round = 0;; ++round) {
                if (round >= sa.max_rounds) { err = true; break; }
                if (++epoch >= 32767) {  // deep-layer tags wrap: clear them
                    __syncthreads();
                    for (int i = tid; i < V; i += NT) s_lab[i] = 0;
                    __syncthreads();
                    epoch = 1;
                }
                if (warp == 0) {
                    halo_seeds(k);
                    u64 Rm[N][RPL], vis[RPL], fr[RPL], ex[RPL];
                    load_masks(Rm);
                    int lmax = 0;
                    bool unreached = false;
#pragma unroll
                    for (int j = 0; j < RPL; ++j) {
                        const int y = lane * RPL + j;
                        ex[j] = s_E[y];
                        fr[j] = s_T[y] | s_seed[y];
                        vis[j] = fr[j];
                        s_layer[1 * TY + y] = fr[j];
                        if (fr[j] & ex[j]) lmax = 1;
                        if (ex[j] & ~vis[j]) unreached = true;
                    }
                    int L = 1;
                    while (__any_sync(0xffffffffu, unreached)) {
                        u64 nf[RPL];
                        expand(Rm, fr, nf);
                        bool any = false;
#pragma unroll
                        for (int j = 0; j < RPL; ++j) {
                            nf[j] &= ~vis[j];
                            any |= nf[j] != 0ull;
                        }
                        if (!__any_sync(0xffffffffu, any)) break;
                        ++L;
                        unreached = false;
#pragma unroll
                        for (int j = 0; j < RPL; ++j) {
                            const int y = lane * RPL + j;
                            vis[j] |= nf[j];
                            fr[j] = nf[j];
                            if (L <= LCAP) {
                                s_layer[L * TY + y] = nf[j];
                            } else {
                                const int tg = deep_tag(epoch, L);
                                for (u64 m = nf[j]; m; m &= m - 1) s_lab[y * TX + __ffsll((long long)m) - 1] = tg;
                            }
                            if (nf[j] & ex[j]) lmax = L;
                            if (ex[j] & ~vis[j]) unreached = true;
                        }
                    }
                    lmax = __reduce_max_sync(0xffffffffu, lmax);
                    if (lane == 0) s_ctl[2] = lmax;
                }
                __syncthreads();
                const int Lmax = s_ctl[2];
                if (Lmax == 0) break;  // no excess vertex reaches T_k: stage done
                ++rounds;
                // layered push, top layer first: a vertex of layer L pushes only to
                // layer L-1 (to T_k from layer 1), so every arc has one writer per step
                for (int L = Lmax; L >= 1; --L) {
                    const int tgL = deep_tag(epoch, L), tgL1 = deep_tag(epoch, L - 1);
                    for (int y = warp; y < TY; y += NW) {
                        u64 P = s_E[y];
                        if (L <= LCAP) P &= s_layer[L * TY + y];
                        if (!P) continue;
#pragma unroll
                        for (int h = 0; h < HW; ++h) {
                            const int lx = lane + 32 * h, ly = y;
                            if (!((P >> lx) & 1ull)) continue;
                            const int i = ly * TX + lx;
                            if (L > LCAP && s_lab[i] != tgL) continue;
                            int e = s_exc[i];
                            if (e <= 0) continue;
                            if (L == 1) {
                                const int tc = s_tcap[i];
                                if (tc > 0) {
                                    const int dl = min(e, tc);
                                    s_tcap[i] = tc - dl;
                                    e -= dl;
                                    flow_acc += dl;
                                    if (tc == dl) atomicAnd(&s_T[ly], ~(1ull << lx));
                                }
#pragma unroll
                                for (int d = 0; d < N; ++d) {
                                    if (e == 0) break;
                                    const int hx = lx + arc_dx(CONN, d), hy = ly + arc_dy(CONN, d);
                                    if (hx >= 0 && hx < TX && hy >= 0 && hy < TY) continue;
                                    const int c = s_cap[d * V + i];
                                    if (c > 0 && s_hl[halo_idx<TX, TY>(hx, hy)] < k) {
                                        const int dl = min(e, c);
                                        s_cap[d * V + i] = c - dl;
                                        e -= dl;
                                        if (c == dl) atomicAnd(&s_R[d * TY + ly], ~(1ull << lx));
                                    }
                                }
                            } else {
#pragma unroll
                                for (int d = 0; d < N; ++d) {
                                    if (e == 0) break;
                                    const int nx = lx + arc_dx(CONN, d), ny = ly + arc_dy(CONN, d);
                                    if (!(nx >= 0 && nx < TX && ny >= 0 && ny < TY)) continue;
                                    const int j = ny * TX + nx;
                                    const int c = s_cap[d * V + i];
                                    if (c <= 0) continue;
                                    const bool below = (L - 1 <= LCAP) ? ((s_layer[(L - 1) * TY + ny] >> nx) & 1ull) != 0
                                                                       : s_lab[j] == tgL1;
                                    if (!below) continue;
                                    const int dl = min(e, c);
                                    s_cap[d * V + i] = c - dl;
                                    const int rc = s_cap[(d ^ 1) * V + j];
                                    s_cap[(d ^ 1) * V + j] = rc + dl;
                                    const int old = atomicAdd(&s_exc[j], dl);
                                    e -= dl;
                                    if (c == dl) atomicAnd(&s_R[d * TY + ly], ~(1ull << lx));
                                    if (rc == 0) atomicOr(&s_R[(d ^ 1) * TY + ny], 1ull << nx);
                                    if (old == 0) atomicOr(&s_E[ny], 1ull << nx);
                                }
                            }
                            s_exc[i] = e;
                            if (e == 0) atomicAnd(&s_E[ly], ~(1ull << lx));
                        }
                    }
                    __syncthreads();
                }
            }
            // the residual graph changed: rebuild the closure and labels of stages <= k
            if (warp == 0) {
#pragma unroll
                for (int j = 0; j < RPL; ++j) Cl[j] = 0;
            }
            for (int k2 = 0;;) {
                if (warp == 0) {
                    closure_extend(k2);
                    const int n2 = next_stage(k2);
                    if (lane == 0) s_ctl[3] = n2;
                }
                __syncthreads();
                write_labels(k2);
                const int n2 = s_ctl[3];
                __syncthreads();
                if (n2 == INT_MAX || n2 > k) break;
                k2 = n2;
            }
        }
        if (kn == INT_MAX) break;
        k = kn;
        __syncthreads();
    }
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < RPL; ++j) s_vis[lane * RPL + j] = Cl[j];
    }
    __syncthreads();

    // ---- write back -------------------------------------------------------------
    int left = 0;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        const int i = tid + q * NT;
        const int lx = i % TX, ly = i / TX;
        const int x = ox + lx, y = oy + ly;
        if (!(x < g.X && y < g.Y)) continue;
        const size_t v = (size_t)y * g.X + x;
        bool perim = false;
#pragma unroll
        for (int d = 0; d < N; ++d) {
            const int nx = lx + arc_dx(CONN, d), ny = ly + arc_dy(CONN, d);
            const int gx = x + arc_dx(CONN, d), gy = y + arc_dy(CONN, d);
            const bool intile = nx >= 0 && nx < TX && ny >= 0 && ny < TY;
            const bool ing = gx >= 0 && gx < g.X && gy >= 0 && gy < g.Y;
            const int c = s_cap[d * V + i];
            if (intile) {
                st.cap[d * n + v] = c;
            } else if (ing) {
                perim = true;
                st.bout[d * n + v] = st.cap[d * n + v] - c;  // flow pushed across the boundary
                st.cap[d * n + v] = c;
            }
        }
        st.tcap[v] = s_tcap[i];
        st.exc[v] = s_exc[i];
        const int lab = ((s_vis[ly] >> lx) & 1ull) ? s_lab[i] : dinf;
        if (perim) st.lab_next[v] = lab;
        else st.lab[v] = lab;
        if (s_exc[i] > 0 && lab < dinf) left = 1;
    }
    left = __syncthreads_or(left);
    unsigned long long f = (unsigned long long)flow_acc;
    for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
    if (lane == 0 && f) atomicAdd(&s_flow, f);
    __syncthreads();
    if (tid == 0) {
        if (s_flow) atomicAdd(st.flow_t, s_flow);
        st.disc[r] = 1;
        st.left_active[r] = (unsigned char)left;
        if (err) atomicExch(&st.ctr[kError], 1);
        atomicAdd(&sa.c64->stages, (unsigned long long)stages);
        atomicAdd(&sa.c64->rounds, (unsigned long long)rounds);
        atomicAdd(&sa.c64->discharges, 1ull);
        const unsigned long long live = (unsigned long long)min(TX, g.X - ox) * min(TY, g.Y - oy);
        atomicAdd(&sa.c64->discharged_vertices, live);
    }
}

template <int CONN, int TX, int TY, int NT>
static cudaError_t launch2d(const Geom &g, const DevState &st, const SweepArgs &sa, cudaStream_t s) {
    using C = Cfg2D<CONN, TX, TY, NT>;
    static bool attr_set = false;
    auto k = ard_discharge2d_kernel<CONN, TX, TY, NT>;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k<<<g.nreg, NT, C::smem, s>>>(g, st, sa);
    return cudaGetLastError();
}

bool discharge2d_supported(int conn, int tx, int ty) {
    return (conn == 4 || conn == 8) && ((tx == 64 && ty == 64) || (tx == 32 && ty == 32));
}

cudaError_t launch_discharge2d(int conn, const Geom &g, const DevState &st, const SweepArgs &sa,
                               cudaStream_t stream) {
    if (conn == 4 && g.tx == 64 && g.ty == 64) return launch2d<4, 64, 64, 512>(g, st, sa, stream);
    if (conn == 8 && g.tx == 64 && g.ty == 64) return launch2d<8, 64, 64, 512>(g, st, sa, stream);
    if (conn == 4 && g.tx == 32 && g.ty == 32) return launch2d<4, 32, 32, 256>(g, st, sa, stream);
    if (conn == 8 && g.tx == 32 && g.ty == 32) return launch2d<8, 32, 32, 256>(g, st, sa, stream);
    return cudaErrorInvalidValue;
}

}  // namespace mf
