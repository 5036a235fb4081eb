// Region discharge of P-ARD for 2D tiles with bit-parallel graph search.
//
// Same computation as ard_discharge.cu (Procedure ARD of Sec. 4.2 with
// Procedure Augment done in synchronous rounds of "BFS from T_k, then a
// layered push from the highest BFS layer down", and the ARD region-relabel
// of Sec. 5.1), organised for a 64- or 32-wide tile:
//
//   * the residual graph of the tile is also kept as bit masks, one 64-bit
//     word per tile row: R_d[y] bit x = [c_f((x,y) -> (x,y)+D(d)) > 0],
//     T[y] bit x = [c_f(v,t) > 0], E[y] bit x = [e_f(v) > 0];
//   * warp 0 (the "graph warp") runs every BFS and reachability flood on these
//     masks: lane l holds rows l*RPL .. l*RPL+RPL-1 in registers; a BFS step is
//     a few shifts/ands per row plus two shuffles for the rows above and below,
//     with no block barrier; floods also close whole row runs at once
//     (Kogge-Stone fill along the row);
//   * all warps do the per-vertex integer work: staging, the layered push,
//     rebuilding the masks from the planes after a push pass, write-back.
//
// Stage checks ("does an excess vertex reach T_k?") use a reachability closure
// C_k extended stage by stage; its increments are the region labels
// d(u) = min{k : u -> T_k}.  Augmentation invalidates the closure; it is then
// rebuilt for the next check, and the labels are recomputed once at the end.
#include <climits>
#include <cstdint>

#include "mf_internal.cuh"

namespace mf {

typedef unsigned long long u64;

#ifdef MF_DIAG
__device__ unsigned long long mf_diag[32];
}  // namespace mf
extern "C" int mf_diag_read(unsigned long long *out, int reset) {
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    if (cudaMemcpyFromSymbol(out, mf::mf_diag, sizeof(unsigned long long) * 32) != cudaSuccess) return 2;
    if (reset) {
        static const unsigned long long z[32] = {0};
        if (cudaMemcpyToSymbol(mf::mf_diag, z, sizeof(z)) != cudaSuccess) return 3;
    }
    return 0;
}
namespace mf {
#endif

template <int CONN, int TX, int TY, int NT>
struct Cfg2D {
    static constexpr int N = CONN;
    static constexpr int V = TX * TY;
    static constexpr int NW = NT / 32;                  // warps
    static constexpr bool PART = TY < 32;               // 32x16 tiles: lanes 16..31 of the graph warp hold no row
    static constexpr int RPL = PART ? 1 : TY / 32;      // rows per lane of the graph warp
    static constexpr int HW = TX / 32;                  // 32-bit halves per row
    static constexpr int HL = 2 * (TX + 2) + 2 * TY;    // halo cells (B^R plus unused corners)
    static constexpr int PER = 2 * TX + 2 * TY;         // perimeter slots: top, bottom, left, right
    // 8-connected 32x32 tiles: four blocks per SM (64 registers, 24 layers kept
    // as masks so that four fit in shared memory; deeper layers use label tags)
    static constexpr bool DENSE = CONN == 8 && TX == 32;
    // 32x16 tiles (128 threads): eight blocks per SM, 16 layers kept as masks
    // at 8-connectivity so that eight fit in shared memory
    static constexpr int LCAP = (DENSE && PART) ? 16 : DENSE ? 24 : 64;  // BFS layers kept as masks
    // resident blocks per SM the registers must allow (64x32 tiles: two, as
    // their shared memory would allow three)
    static constexpr int MINB = PART ? 8 : DENSE ? 4 : (CONN == 4 && TX == 32) ? 4 : (TX * TY == 2048) ? 2 : 1;
    static constexpr size_t smem = (size_t)(N + 3) * V * 4                  // cap, tcap, exc, lab
                                   + (size_t)(N + 4) * TY * 8               // R[N], T, E, inc, vis
                                   + (size_t)(LCAP + 1) * TY * 8            // BFS layers 1..LCAP
                                   + (size_t)(HL + PER) * 4 + TY + 64;      // halo labels, hmin, dirty rows
    static_assert(TX == 32 || TX == 64, "row width must be 32 or 64");
    static_assert((TY % 32 == 0 || (TY == 16 && TX == 32)) && TY <= 64 && V % NT == 0 && NT % 32 == 0,
                  "tile/threads mismatch");
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
__device__ __forceinline__ void discharge2d_region(const Geom &g, const DevState &st, const SweepArgs &sa,
                                                   const int r, unsigned long long *mbar, unsigned &mphase) {
    using C = Cfg2D<CONN, TX, TY, NT>;
    constexpr int N = C::N, V = C::V, RPL = C::RPL, NW = C::NW, HW = C::HW, LCAP = C::LCAP;
    extern __shared__ __align__(16) unsigned char smraw[];
    int *s_cap = (int *)smraw;            // [N][V] residual of arc i -> i + D(d)
    int *s_tcap = s_cap + N * V;          // [V]
    int *s_exc = s_tcap + V;              // [V]
    int *s_lab = s_exc + V;               // [V] region label (deep BFS layers: negative tags)
    u64 *s_R = (u64 *)(s_lab + V);        // [N][TY] residual masks
    u64 *s_T = s_R + N * TY;              // [TY] residual arc to t
    u64 *s_E = s_T + TY;                  // [TY] positive excess
    u64 *s_inc = s_E + TY;                // [TY] vertices that joined the closure
    u64 *s_vis = s_inc + TY;              // [TY] final closure (during Augment rounds: excess received)
    u64 *s_layer = s_vis + TY;            // [LCAP+1][TY] BFS layers
    int *s_hl = (int *)(s_layer + (LCAP + 1) * TY);  // [HL] labels of B^R
    int *s_hmin = s_hl + C::HL;           // [PER] min label over residual boundary arcs of a perimeter vertex
    unsigned char *s_dirty = (unsigned char *)(s_hmin + C::PER);  // [TY] rows whose planes changed
    __shared__ int s_ctl[4];
    __shared__ unsigned long long s_flow;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // does this lane of the graph warp hold tile rows (all do unless the tile has 16 rows)
    const bool lrow = !C::PART || lane < TY;
    DIAG_DECL
    const long long diag_t0 = clock64();
    (void)diag_t0;
    const int rx = r % g.RX, ry = r / g.RX;
    const int ox = rx * TX, oy = ry * TY;
    const size_t n = (size_t)g.n;
    const int dinf = g.dinf;
    if (tid == 0) s_flow = 0;

    // rebuild the row masks from the planes (all threads; a warp covers 32
    // consecutive vertices of one row, so one ballot gives half a row word);
    // with only_round, just the rows the last Augment round changed (s_dirty 2)
    auto rebuild_masks = [&](bool only_round) {
        for (int i = tid; i < V; i += NT) {
            const int lx = i % TX, ly = i / TX;
            if (only_round && s_dirty[ly] != 2) continue;  // the same row for the whole warp
            const int hw = (ly * 2 + (lx >> 5));
#pragma unroll
            for (int d = 0; d < N; ++d) {
                const unsigned b = __ballot_sync(0xffffffffu, s_cap[d * V + i] > 0);
                if (lane == 0) ((unsigned *)s_R)[d * TY * 2 + hw] = b;
            }
            const unsigned bt = __ballot_sync(0xffffffffu, s_tcap[i] > 0);
            const unsigned be = __ballot_sync(0xffffffffu, s_exc[i] > 0);
            if (lane == 0) {
                ((unsigned *)s_T)[hw] = bt;
                ((unsigned *)s_E)[hw] = be;
            }
        }
    };
    // perimeter slot p -> tile coordinates (top row, bottom row, left column, right column)
    auto per_xy = [](int p, int &x, int &y) {
        if (p < TX) { x = p; y = 0; }
        else if (p < 2 * TX) { x = p - TX; y = TY - 1; }
        else if (p < 2 * TX + TY) { x = 0; y = p - 2 * TX; }
        else { x = TX - 1; y = p - 2 * TX - TY; }
    };
    // hmin[p] = min{d(w) : residual arc from the perimeter vertex to w in B^R}
    // with only_round, just the slots whose row the last Augment round changed
    // (a boundary arc's residual changes only by a push of its own cell)
    auto rebuild_hmin = [&](bool only_round) {
        for (int p = tid; p < C::PER; p += NT) {
            int x, y;
            per_xy(p, x, y);
            if (only_round && s_dirty[y] != 2) continue;
            int m = INT_MAX;
#pragma unroll
            for (int d = 0; d < N; ++d) {
                const int hx = x + arc_dx(CONN, d), hy = y + arc_dy(CONN, d);
                if (hx >= 0 && hx < TX && hy >= 0 && hy < TY) continue;
                if (s_cap[d * V + y * TX + x] > 0) m = min(m, s_hl[halo_idx<TX, TY>(hx, hy)]);
            }
            s_hmin[p] = m;
        }
    };

    // ---- stage the tile --------------------------------------------------------
    const bool full = ox + TX <= g.X && oy + TY <= g.Y;
    // bulk copies need every row on a 16-byte boundary; planes in host memory
    // are read with plain loads
    const bool vec = full && (g.X % 4) == 0 && !st.host;
    if (vec) {
        // one bulk copy per row of every plane (cap[N], tcap, exc are adjacent in
        // shared memory) against the block's transaction barrier, spread over
        // all threads; the labels start at 0 and the halo is gathered meanwhile
        fence_proxy_async_smem();
        if (tid == 0) mbar_arrive_expect_tx(mbar, (unsigned)((N + 2) * V * 4));
        __syncthreads();  // earlier accesses of the planes and the byte count precede the copies
        for (int c = tid; c < (N + 2) * TY; c += NT) {
            const int p = c / TY, ly = c % TY;
            const int *plane = p < N ? st.cap + (size_t)p * n : p == N ? st.tcap : st.exc;
            bulk_g2s(s_cap + p * V + ly * TX, plane + (size_t)(oy + ly) * g.X + ox, TX * 4, mbar);
        }
        for (int i4 = tid; i4 < V / 4; i4 += NT) *(int4 *)&s_lab[i4 * 4] = make_int4(0, 0, 0, 0);
    } else {
        for (int i = tid; i < V; i += NT) {
            const int lx = i % TX, ly = i / TX;
            const int x = ox + lx, y = oy + ly;
            const bool in = x < g.X && y < g.Y;
            const size_t v = (size_t)y * g.X + x;
#pragma unroll
            for (int d = 0; d < N; ++d) s_cap[d * V + i] = in ? st.cap[d * n + v] : 0;
            s_tcap[i] = in ? st.tcap[v] : 0;
            s_exc[i] = in ? st.exc[v] : 0;
            s_lab[i] = 0;
        }
    }
    for (int y = tid; y < TY; y += NT) s_dirty[y] = 0;
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
    if (TX == 32) {  // upper halves of the row words are never written by the ballots
        for (int w = tid; w < (N + 2) * TY; w += NT) ((unsigned *)s_R)[w * 2 + 1] = 0;
    }
    if (vec) {
        bool landed = mbar_wait(mbar, mphase);
        if (!landed) landed = mbar_wait(mbar, mphase);  // once more (bounded) before giving up
        mphase ^= 1u;
        if (__syncthreads_or(!landed)) {  // never expected: report and leave the region untouched
            if (tid == 0) atomicExch(&st.ctr[kError], 2);
            return;
        }
    }
    __syncthreads();
    rebuild_masks(false);
    rebuild_hmin(false);
    __syncthreads();
    DIAG_LAP(0);

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
    // seed rows of T_k: vertices with a residual arc to t, or to w in B^R with d(w) < k
    auto seed_rows = [&](int k, u64 (&sd)[RPL]) {
        u64 top = 0, bot = 0;
#pragma unroll
        for (int h = 0; h < HW; ++h) {
            const int x = lane + 32 * h;
            top |= (u64)__ballot_sync(0xffffffffu, s_hmin[x] < k) << (32 * h);
            bot |= (u64)__ballot_sync(0xffffffffu, s_hmin[TX + x] < k) << (32 * h);
        }
        unsigned lft[RPL], rgt[RPL];
#pragma unroll
        for (int h = 0; h < RPL; ++h) {
            const int y = lane + 32 * h;
            lft[h] = __ballot_sync(0xffffffffu, y < TY && s_hmin[2 * TX + y] < k);
            rgt[h] = __ballot_sync(0xffffffffu, y < TY && s_hmin[2 * TX + TY + y] < k);
        }
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int y = lane * RPL + j;
            u64 s = 0;
            if (lrow) {
                s = s_T[y];
                s |= (u64)((lft[y >> 5] >> (y & 31)) & 1u);
                s |= (u64)((rgt[y >> 5] >> (y & 31)) & 1u) << (TX - 1);
                if (y == 0) s |= top;
                if (y == TY - 1) s |= bot;
            }
            sd[j] = s;
        }
    };
    auto load_masks = [&](u64 (&Rm)[N][RPL]) {
#pragma unroll
        for (int j = 0; j < RPL; ++j)
#pragma unroll
            for (int d = 0; d < N; ++d) Rm[d][j] = lrow ? s_R[d * TY + lane * RPL + j] : 0ull;
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
    // closure Cl := Cl U {u : u -> sd} (residual reachability); increments to s_inc
    u64 Cl[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) Cl[j] = 0;
    auto flood = [&](const u64 (&sd)[RPL]) {
        u64 Rm[N][RPL], fr[RPL], inc[RPL];
        load_masks(Rm);
        bool any = false;
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const u64 f = row_fill(sd[j] & ~Cl[j], Rm[0][j] & ~Cl[j], Rm[1][j] & ~Cl[j]);
            Cl[j] |= f;
            inc[j] = f;
            fr[j] = f;
            any |= f != 0ull;
        }
        while (__any_sync(0xffffffffu, any)) {
            u64 nf[RPL];
            expand(Rm, fr, nf);
            any = false;
            DIAG_ADD(3, 1);
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                const u64 f = row_fill(nf[j] & ~Cl[j], Rm[0][j] & ~Cl[j], Rm[1][j] & ~Cl[j]);
                Cl[j] |= f;
                inc[j] |= f;
                fr[j] = f;
                any |= f != 0ull;
            }
        }
        if (lrow) {
#pragma unroll
            for (int j = 0; j < RPL; ++j) s_inc[lane * RPL + j] = inc[j];
        }
    };
    auto closure_meets_excess = [&]() -> bool {
        bool m = false;
#pragma unroll
        for (int j = 0; j < RPL; ++j) m |= lrow && (Cl[j] & s_E[lane * RPL + j]) != 0ull;
        return __any_sync(0xffffffffu, m);
    };
    // all threads: label the vertices of s_inc with k
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

    const int klimit = sa.partial ? (sa.sweep_dev ? *sa.sweep_dev : sa.sweep) : INT_MAX;
    long long flow_acc = 0;
    int rounds = 0, stages = 0, epoch = 0;
    bool err = false, any_aug = false;
    bool cl_valid = true;  // warp 0: Cl is the closure of T_k on the current graph (empty at start)

    // ---- ARD stages ------------------------------------------------------------
    for (int k = 0;;) {
        DIAG_MARK();
        if (warp == 0) {
            DIAG_ADD(2, 1);
            u64 sd[RPL];
            seed_rows(k, sd);
            if (!cl_valid) {
#pragma unroll
                for (int j = 0; j < RPL; ++j) Cl[j] = 0;
                cl_valid = true;
            }
            flood(sd);
            const bool reach = closure_meets_excess();
            const int kn = next_stage(k);
            if (lane == 0) {
                s_ctl[0] = reach;
                s_ctl[1] = kn;
            }
        }
        __syncthreads();
        DIAG_LAP(1);
        const int reach = s_ctl[0], kn = s_ctl[1];
        if (!any_aug) write_labels(k);  // labels stay exact until the first augmentation
        const bool aug = k <= klimit && !err;
        if (aug) ++stages;
        if (aug && reach) {
            any_aug = true;
            // Augment(R, T_k): rounds of exact BFS + layered push
            for (int round = 0;; ++round) {
                if (round >= sa.max_rounds) { err = true; break; }
                if (++epoch >= 32767) {  // deep-layer tags wrap: clear them
                    __syncthreads();
                    for (int i = tid; i < V; i += NT) s_lab[i] = 0;
                    __syncthreads();
                    epoch = 1;
                }
                DIAG_MARK();
                if (warp == 0) {
                    DIAG_ADD(5, 1);
                    u64 Rm[N][RPL], vis[RPL], fr[RPL], want[RPL];
                    load_masks(Rm);
                    seed_rows(k, fr);
                    int lmax = 0;
                    bool pending = false;
#pragma unroll
                    for (int j = 0; j < RPL; ++j) {
                        const int y = lane * RPL + j;
                        // excess that can reach T_k lies inside the (older) closure
                        const u64 ex = lrow ? s_E[y] & Cl[j] : 0ull;
                        vis[j] = fr[j];
                        if (lrow) {
                            s_layer[1 * TY + y] = fr[j];
                            s_vis[y] = 0ull;  // vertices that receive excess in this round's push
                        }
                        if (fr[j] & ex) lmax = 1;
                        want[j] = ex & ~vis[j];
                        pending |= want[j] != 0ull;
                    }
                    int L = 1;
                    while (__any_sync(0xffffffffu, pending)) {
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
                        pending = false;
#pragma unroll
                        for (int j = 0; j < RPL; ++j) {
                            const int y = lane * RPL + j;
                            vis[j] |= nf[j];
                            fr[j] = nf[j];
                            if (L <= LCAP) {
                                if (lrow) s_layer[L * TY + y] = nf[j];
                            } else {
                                const int tg = deep_tag(epoch, L);
                                for (u64 m = nf[j]; m; m &= m - 1) s_lab[y * TX + __ffsll((long long)m) - 1] = tg;
                            }
                            if (nf[j] & want[j]) lmax = L;
                            want[j] &= ~nf[j];
                            pending |= want[j] != 0ull;
                        }
                    }
                    lmax = __reduce_max_sync(0xffffffffu, lmax);
                    if (lane == 0) s_ctl[2] = lmax;
                    DIAG_ADD(6, L);
                }
                __syncthreads();
                DIAG_LAP(4);
                const int Lmax = s_ctl[2];
                if (Lmax == 0) break;  // no excess vertex reaches T_k: stage done
                ++rounds;
                // layered push, top layer first: a vertex of layer L pushes only to
                // layer L-1 (to T_k from layer 1), so every arc has one writer per step.
                // The masks R_d are exact for the arcs from layer L to L-1 until layer L
                // pushes, so A_d = R_d & (layer L-1 seen through arc d) lists the
                // admissible arcs of a whole row at once.  Only vertices that had
                // excess when the round began (s_E) or received some in an earlier
                // step of it (s_vis) can push, so rows without such a vertex of
                // layer L are passed over.
                u64 *s_recv = s_vis;
                for (int L = Lmax; L >= 1; --L) {
                    const int tgL = deep_tag(epoch, L), tgL1 = deep_tag(epoch, L - 1);
                    const bool lo_mask = L - 1 <= LCAP;
                    for (int y = warp; y < TY; y += NW) {
                        const u64 P = (L <= LCAP ? s_layer[L * TY + y] : ~0ull) & (s_E[y] | s_recv[y]);
                        if (!P) continue;
                        u64 A[N];
                        if (L > 1 && lo_mask) {
                            const u64 *lay = s_layer + (L - 1) * TY;
                            const u64 la = y > 0 ? lay[y - 1] : 0ull, l0 = lay[y], lb = y < TY - 1 ? lay[y + 1] : 0ull;
#pragma unroll
                            for (int d = 0; d < N; ++d) {
                                const int dx = arc_dx(CONN, d), dy = arc_dy(CONN, d);
                                const u64 src = dy < 0 ? la : dy > 0 ? lb : l0;
                                const u64 sh = dx > 0 ? (src >> 1) : dx < 0 ? (src << 1) : src;
                                A[d] = s_R[d * TY + y] & sh;
                            }
                        }
                        bool pushed = false;
#pragma unroll
                        for (int h = 0; h < HW; ++h) {
                            const int lx = lane + 32 * h, ly = y;
                            if (!((P >> lx) & 1ull)) continue;
                            const int i = ly * TX + lx;
                            if (L > LCAP && s_lab[i] != tgL) continue;
                            int e = s_exc[i];
                            if (e <= 0) continue;
                            const int e0 = e;
                            if (L == 1) {
                                const int tc = s_tcap[i];
                                if (tc > 0) {
                                    const int dl = min(e, tc);
                                    s_tcap[i] = tc - dl;
                                    e -= dl;
                                    flow_acc += dl;
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
                                    }
                                }
                            } else {
#pragma unroll
                                for (int d = 0; d < N; ++d) {
                                    if (e == 0) break;
                                    const int nx = lx + arc_dx(CONN, d), ny = ly + arc_dy(CONN, d);
                                    bool adm;
                                    if (lo_mask) {
                                        adm = (A[d] >> lx) & 1ull;
                                    } else {
                                        adm = nx >= 0 && nx < TX && ny >= 0 && ny < TY &&
                                              s_lab[ny * TX + nx] == tgL1 && s_cap[d * V + i] > 0;
                                    }
                                    if (!adm) continue;
                                    const int j = ny * TX + nx;
                                    const int c = s_cap[d * V + i];
                                    const int dl = min(e, c);
                                    s_cap[d * V + i] = c - dl;
                                    s_cap[(d ^ 1) * V + j] += dl;
                                    atomicAdd(&s_exc[j], dl);
                                    atomicOr((unsigned *)&s_recv[ny] + (nx >> 5), 1u << (nx & 31));
                                    e -= dl;
                                }
                            }
                            s_exc[i] = e;
                            pushed |= e != e0;
                        }
                        if (__any_sync(0xffffffffu, pushed) && lane < 3) {
                            const int yy = y - 1 + lane;
                            if (yy >= 0 && yy < TY) s_dirty[yy] = 2;  // changed in this round
                        }
                    }
                    __syncthreads();
                }
                rebuild_masks(true);  // a push changes rows y-1..y+1 only
                rebuild_hmin(true);
                __syncthreads();
                for (int y = tid; y < TY; y += NT)
                    if (s_dirty[y] == 2) s_dirty[y] = 1;
                DIAG_LAP(7);
                DIAG_ADD(8, Lmax);
            }
            if (warp == 0) cl_valid = false;  // the residual graph changed
        }
        if (kn == INT_MAX) break;
        // nothing left to learn: labels are recomputed at the end anyway
        if (any_aug && (kn > klimit || err)) break;
        k = kn;
        __syncthreads();
    }

    // ---- region-relabel after augmentation: d(u) = min{k : u -> T_k} -------------
    if (any_aug) {
        DIAG_MARK();
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int j = 0; j < RPL; ++j) Cl[j] = 0;
        }
        for (int k2 = 0;;) {
            if (warp == 0) {
                DIAG_ADD(2, 1);
                u64 sd[RPL];
                seed_rows(k2, sd);
                flood(sd);
                const int n2 = next_stage(k2);
                if (lane == 0) s_ctl[3] = n2;
            }
            __syncthreads();
            write_labels(k2);
            const int n2 = s_ctl[3];
            __syncthreads();
            if (n2 == INT_MAX) break;
            k2 = n2;
        }
        DIAG_LAP(9);
    }
    if (warp == 0 && lrow) {
#pragma unroll
        for (int j = 0; j < RPL; ++j) s_vis[lane * RPL + j] = Cl[j];
    }
    __syncthreads();
    DIAG_MARK();

    // ---- write back: planes of rows that changed; labels and boundary flows always
    int left = 0;
    for (int i = tid; i < V; i += NT) {
        const int lx = i % TX, ly = i / TX;
        const int x = ox + lx, y = oy + ly;
        if (!(x < g.X && y < g.Y)) continue;
        const size_t v = (size_t)y * g.X + x;
        const bool dirty = s_dirty[ly] != 0;
        bool perim = false;
#pragma unroll
        for (int d = 0; d < N; ++d) {
            const int nx = lx + arc_dx(CONN, d), ny = ly + arc_dy(CONN, d);
            const int gx = x + arc_dx(CONN, d), gy = y + arc_dy(CONN, d);
            const bool intile = nx >= 0 && nx < TX && ny >= 0 && ny < TY;
            const bool ing = gx >= 0 && gx < g.X && gy >= 0 && gy < g.Y;
            if (intile) {
                if (dirty) st.cap[d * n + v] = s_cap[d * V + i];
            } else if (ing) {
                perim = true;
                if (dirty) {
                    const int c = s_cap[d * V + i];
                    st.bout[d * n + v] = st.cap[d * n + v] - c;  // flow pushed across the boundary
                    st.cap[d * n + v] = c;
                } else {
                    st.bout[d * n + v] = 0;
                }
            }
        }
        if (dirty) {
            st.tcap[v] = s_tcap[i];
            st.exc[v] = s_exc[i];
        }
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
        DIAG_LAP(10);
        DIAG_ADD(11, clock64() - diag_t0);
        DIAG_ADD(12, 1);
        DIAG_FLUSH();
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

// one block per region of one grid; regions without active vertices are skipped (Sec. 5.3)
template <int CONN, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, (Cfg2D<CONN, TX, TY, NT>::MINB)) ard_discharge2d_kernel(const Geom g, const DevState st, const SweepArgs sa) {
    const int r = blockIdx.x;
    if (!st.active[r]) return;
    __shared__ __align__(8) unsigned long long s_mbar;
    if (threadIdx.x == 0) mbar_init(&s_mbar, 1);
    __syncthreads();
    unsigned phase = 0;
    discharge2d_region<CONN, TX, TY, NT>(g, st, sa, r, &s_mbar, phase);
}

// persistent blocks over a work queue of (instance, region) items of a batch
template <int CONN, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, (Cfg2D<CONN, TX, TY, NT>::MINB))
ard_discharge2d_batch_kernel(const Inst *__restrict__ insts, const int2 *__restrict__ items, const int *count,
                             int *head, const SweepArgs sa) {
    __shared__ int s_it;
    __shared__ __align__(8) unsigned long long s_mbar;
    if (threadIdx.x == 0) mbar_init(&s_mbar, 1);
    unsigned phase = 0;
    for (;;) {
        __syncthreads();  // the previous item is done with s_it and the shared planes
        if (threadIdx.x == 0) s_it = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_it;
        if (it >= *count) break;
        const int2 w = items[it];
        const Inst &I = insts[w.x];
        SweepArgs a = sa;
        a.c64 = I.c64;
        discharge2d_region<CONN, TX, TY, NT>(I.g, I.st, a, w.y, &s_mbar, phase);
    }
}

template <int CONN, int TX, int TY, int NT>
static cudaError_t launch2d_batch(const Inst *insts, const int2 *items, const int *count, int *head,
                                  const SweepArgs &sa, int blocks, cudaStream_t s) {
    using C = Cfg2D<CONN, TX, TY, NT>;
    auto k = ard_discharge2d_batch_kernel<CONN, TX, TY, NT>;
    {
        const cudaError_t e_at = ensure_smem_attr((const void *)k, (int)C::smem);
        if (e_at != cudaSuccess) return e_at;
    }
    const int resident = device_sms() * C::MINB;  // persistent blocks: at least as many as can be resident
    k<<<blocks > resident ? blocks : resident, NT, C::smem, s>>>(insts, items, count, head, sa);
    return cudaGetLastError();
}

template <int CONN, int TX, int TY, int NT>
static cudaError_t launch2d(const Geom &g, const DevState &st, const SweepArgs &sa, cudaStream_t s) {
    using C = Cfg2D<CONN, TX, TY, NT>;
    auto k = ard_discharge2d_kernel<CONN, TX, TY, NT>;
    {
        const cudaError_t e_at = ensure_smem_attr((const void *)k, (int)C::smem);
        if (e_at != cudaSuccess) return e_at;
    }
    k<<<g.nreg, NT, C::smem, s>>>(g, st, sa);
    return cudaGetLastError();
}

bool discharge2d_supported(int conn, int tx, int ty) {
    return (conn == 4 || conn == 8) &&
           ((tx == 64 && ty == 64) || (tx == 32 && ty == 32) || (tx == 64 && ty == 32) || (tx == 32 && ty == 16));
}

cudaError_t launch_discharge2d_batch(int conn, int tx, int ty, const Inst *insts, const int2 *items,
                                     const int *count, int *head, const SweepArgs &sa, int blocks,
                                     cudaStream_t stream) {
    if (conn == 4 && tx == 64 && ty == 64) return launch2d_batch<4, 64, 64, 512>(insts, items, count, head, sa, blocks, stream);
    if (conn == 8 && tx == 64 && ty == 64) return launch2d_batch<8, 64, 64, 512>(insts, items, count, head, sa, blocks, stream);
    if (conn == 4 && tx == 32 && ty == 32) return launch2d_batch<4, 32, 32, 256>(insts, items, count, head, sa, blocks, stream);
    if (conn == 8 && tx == 32 && ty == 32) return launch2d_batch<8, 32, 32, 256>(insts, items, count, head, sa, blocks, stream);
    if (conn == 4 && tx == 64 && ty == 32) return launch2d_batch<4, 64, 32, 256>(insts, items, count, head, sa, blocks, stream);
    if (conn == 8 && tx == 64 && ty == 32) return launch2d_batch<8, 64, 32, 256>(insts, items, count, head, sa, blocks, stream);
    if (conn == 4 && tx == 32 && ty == 16) return launch2d_batch<4, 32, 16, 128>(insts, items, count, head, sa, blocks, stream);
    if (conn == 8 && tx == 32 && ty == 16) return launch2d_batch<8, 32, 16, 128>(insts, items, count, head, sa, blocks, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_discharge2d(int conn, const Geom &g, const DevState &st, const SweepArgs &sa,
                               cudaStream_t stream) {
    if (conn == 4 && g.tx == 64 && g.ty == 64) return launch2d<4, 64, 64, 512>(g, st, sa, stream);
    if (conn == 8 && g.tx == 64 && g.ty == 64) return launch2d<8, 64, 64, 512>(g, st, sa, stream);
    if (conn == 4 && g.tx == 32 && g.ty == 32) return launch2d<4, 32, 32, 256>(g, st, sa, stream);
    if (conn == 8 && g.tx == 32 && g.ty == 32) return launch2d<8, 32, 32, 256>(g, st, sa, stream);
    if (conn == 4 && g.tx == 64 && g.ty == 32) return launch2d<4, 64, 32, 256>(g, st, sa, stream);
    if (conn == 8 && g.tx == 64 && g.ty == 32) return launch2d<8, 64, 32, 256>(g, st, sa, stream);
    if (conn == 4 && g.tx == 32 && g.ty == 16) return launch2d<4, 32, 16, 128>(g, st, sa, stream);
    if (conn == 8 && g.tx == 32 && g.ty == 16) return launch2d<8, 32, 16, 128>(g, st, sa, stream);
    return cudaErrorInvalidValue;
}

}  // namespace mf
