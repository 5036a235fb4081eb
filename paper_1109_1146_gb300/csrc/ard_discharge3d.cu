// Region discharge of P-ARD for 3D 6-connected tiles with bit-parallel graph
// search.
//
// The same computation as ard_discharge.cu and ard_discharge2d.cu (Procedure
// ARD of Sec. 4.2, Procedure Augment in synchronous rounds of "exact BFS from
// T_k, then a layered push from the highest BFS layer down", the ARD
// region-relabel of Sec. 5.1), for tiles 32 voxels wide in x:
//
//   * a "row" is the run of 32 voxels along x at one (y, z) of the tile, row
//     index rho = z * TY + y; every mask holds one 32-bit word per row:
//     R_d[rho] bit x = [c_f(v -> v + D(d)) > 0] for the six arcs
//     d = +x, -x, +y, -y, +z, -z, T[rho] = [c_f(v,t) > 0], E[rho] = [e_f(v) > 0];
//   * warp 0 (the graph warp) runs every BFS and reachability flood on these
//     masks: lane l holds rows l*RPL .. l*RPL+RPL-1; a step shifts a word for
//     +-x, takes the neighbouring row for +-y (a shuffle across one lane at
//     the ends of a lane's rows) and the row TY away for +-z (a shuffle across
//     TY/RPL lanes); floods close whole x-runs at once (Kogge-Stone fill);
//   * every arc leaving the tile ends in its own halo cell (six faces), so the
//     boundary of T_k is a table over halo cells: hm[h] = d(h) if the arc
//     into h has residual capacity, else infinity;
//   * all warps do the per-vertex integer work: staging, the layered push,
//     rebuilding the masks after a push pass, write-back.
#include <climits>
#include <cstdint>

#include "mf_internal.cuh"

namespace mf {

typedef unsigned int u32;

#ifdef MF_DIAG
__device__ unsigned long long mf_diag3[32];
}  // namespace mf
extern "C" int mf_diag3_read(unsigned long long *out, int reset) {
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    if (cudaMemcpyFromSymbol(out, mf::mf_diag3, sizeof(unsigned long long) * 32) != cudaSuccess) return 2;
    if (reset) {
        static const unsigned long long z[32] = {0};
        if (cudaMemcpyToSymbol(mf::mf_diag3, z, sizeof(z)) != cudaSuccess) return 3;
    }
    return 0;
}
namespace mf {
#define mf_diag mf_diag3
#endif

template <int TY, int TZ, int NT>
struct Cfg3D {
    static constexpr int TX = 32, N = 6;
    static constexpr int NR = TY * TZ;            // rows of the tile
    static constexpr int V = TX * NR;             // voxels
    static constexpr int NW = NT / 32;            // warps
    static constexpr bool PART = NR < 32;         // 16-row tiles: lanes 16..31 of the graph warp hold no row
    static constexpr int RPL = PART ? 1 : NR / 32;  // rows per lane of the graph warp
    static constexpr int LZ = TY / RPL;           // lanes between rows rho and rho + TY
    // halo faces: -x, +x (one cell per row), -y, +y (TX per z), -z, +z (TX per y)
    static constexpr int B_MX = 0, B_PX = NR, B_MY = 2 * NR, B_PY = 2 * NR + TX * TZ;
    static constexpr int B_MZ = 2 * NR + 2 * TX * TZ, B_PZ = B_MZ + TX * TY;
    static constexpr int HL = B_PZ + TX * TY;     // halo cells = arcs leaving the tile
    static constexpr int LCAP = 32;               // BFS layers kept as masks
    // resident blocks per SM the registers must allow (shared memory allows
    // eight 16-row tiles at 128 threads, four 32x8x4 tiles, two 32x8x8 tiles,
    // one 32x16x8 tile)
    static constexpr int MINB = NR == 16 ? 8 : NR == 32 ? 4 : NR == 64 ? 2 : 1;
    static constexpr size_t smem = (size_t)(N + 3) * V * 4           // cap, tcap, exc, lab
                                   + (size_t)(N + 4) * NR * 4        // R[N], T, E, inc, vis
                                   + (size_t)(LCAP + 1) * NR * 4     // BFS layers 1..LCAP
                                   + (size_t)2 * HL * 4 + NR + 64;   // halo labels, hm, dirty rows
    static_assert((NR % 32 == 0 || NR == 16) && TY % RPL == 0 && V % NT == 0 && NT % 32 == 0, "tile/threads mismatch");
};

// Kogge-Stone fill inside one 32-bit row: x joins if x+1 is in g and pl[x]
// (arc x -> x+1), or x-1 is in g and pr[x] (arc x -> x-1), repeatedly.
__device__ __forceinline__ u32 row_fill32(u32 g, u32 pl, u32 pr) {
    u32 a = g, p = pl;
    a |= p & (a >> 1);  p &= p >> 1;
    a |= p & (a >> 2);  p &= p >> 2;
    a |= p & (a >> 4);  p &= p >> 4;
    a |= p & (a >> 8);  p &= p >> 8;
    a |= p & (a >> 16);
    u32 b = g;
    p = pr;
    b |= p & (b << 1);  p &= p << 1;
    b |= p & (b << 2);  p &= p << 2;
    b |= p & (b << 4);  p &= p << 4;
    b |= p & (b << 8);  p &= p << 8;
    b |= p & (b << 16);
    return a | b;
}

__device__ __forceinline__ int deep_tag3(int epoch, int L) { return ~((epoch << 16) | L); }

// halo cell of the arc d leaving the tile at tile voxel (lx, ly, lz)
template <int TY, int TZ>
__device__ __forceinline__ int halo3(int d, int lx, int ly, int lz) {
    constexpr int TX = 32, NR = TY * TZ;
    constexpr int B_MX = 0, B_PX = NR, B_MY = 2 * NR, B_PY = 2 * NR + TX * TZ;
    constexpr int B_MZ = 2 * NR + 2 * TX * TZ, B_PZ = B_MZ + TX * TY;
    switch (d) {
        case 0: return B_PX + lz * TY + ly;
        case 1: return B_MX + lz * TY + ly;
        case 2: return B_PY + lz * TX + lx;
        case 3: return B_MY + lz * TX + lx;
        case 4: return B_PZ + ly * TX + lx;
        default: return B_MZ + ly * TX + lx;
    }
}

// tile voxel and arc of halo cell h (inverse of halo3); the cell itself lies
// one step along the arc
template <int TY, int TZ>
__device__ __forceinline__ void halo3_src(int h, int &lx, int &ly, int &lz, int &d) {
    constexpr int TX = 32, NR = TY * TZ;
    if (h < NR) { lx = 0; ly = h % TY; lz = h / TY; d = 1; return; }
    if (h < 2 * NR) { const int q = h - NR; lx = TX - 1; ly = q % TY; lz = q / TY; d = 0; return; }
    int q = h - 2 * NR;
    if (q < TX * TZ) { lx = q % TX; lz = q / TX; ly = 0; d = 3; return; }
    q -= TX * TZ;
    if (q < TX * TZ) { lx = q % TX; lz = q / TX; ly = TY - 1; d = 2; return; }
    q -= TX * TZ;
    if (q < TX * TY) { lx = q % TX; ly = q / TX; lz = 0; d = 5; return; }
    q -= TX * TY;
    lx = q % TX; ly = q / TX; lz = TZ - 1; d = 4;
}

template <int TY, int TZ, int NT>
__device__ __forceinline__ void discharge3d_region(const Geom &g, const DevState &st, const SweepArgs &sa,
                                                   const int r, unsigned long long *mbar, unsigned &mphase) {
    using C = Cfg3D<TY, TZ, NT>;
    constexpr int TX = 32, N = 6, V = C::V, NR = C::NR, RPL = C::RPL, NW = C::NW, LCAP = C::LCAP, LZ = C::LZ;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smraw[];
    int *s_cap = (int *)smraw;              // [N][V] residual of arc i -> i + D(d)
    int *s_tcap = s_cap + N * V;            // [V]
    int *s_exc = s_tcap + V;                // [V]
    int *s_lab = s_exc + V;                 // [V] region label (deep BFS layers: negative tags)
    u32 *s_R = (u32 *)(s_lab + V);          // [N][NR] residual masks
    u32 *s_T = s_R + N * NR;                // [NR]
    u32 *s_E = s_T + NR;                    // [NR]
    u32 *s_inc = s_E + NR;                  // [NR]
    u32 *s_vis = s_inc + NR;                // [NR] final closure (during Augment rounds: excess received)
    u32 *s_layer = s_vis + NR;              // [LCAP+1][NR]
    int *s_hl = (int *)(s_layer + (LCAP + 1) * NR);  // [HL] labels of B^R
    int *s_hm = s_hl + C::HL;               // [HL] label of the halo cell if its arc is residual, else INT_MAX
    unsigned char *s_dirty = (unsigned char *)(s_hm + C::HL);  // [NR] rows whose planes changed
    __shared__ int s_ctl[4];
    __shared__ unsigned long long s_flow;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // does this lane of the graph warp hold tile rows (all do unless the tile has 16 rows)
    const bool lrow = !C::PART || lane < NR;
    DIAG_DECL
    const long long diag_t0 = clock64();
    (void)diag_t0;
    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    const int ox = rx * TX, oy = ry * TY, oz = rz * TZ;
    const size_t n = (size_t)g.n;
    const int dinf = g.dinf;
    if (tid == 0) s_flow = 0;

    // voxel index i = rho * TX + x, rho = z * TY + y; plane offset of each arc
    auto arc_off = [](int d) -> int {
        return d == 0 ? 1 : d == 1 ? -1 : d == 2 ? TX : d == 3 ? -TX : d == 4 ? TX * TY : -TX * TY;
    };
    // does arc d from row rho stay in the tile along y / z (x handled by the word shifts)
    auto row_has = [](int d, int rho) -> bool {
        const int y = rho % TY, z = rho / TY;
        return d == 2 ? y < TY - 1 : d == 3 ? y > 0 : d == 4 ? z < TZ - 1 : d == 5 ? z > 0 : true;
    };
    // with only_round, just the rows the last Augment round changed (s_dirty 2)
    auto rebuild_masks = [&](bool only_round) {
        for (int i = tid; i < V; i += NT) {
            const int rho = i / TX;
            if (only_round && s_dirty[rho] != 2) continue;  // the same row for the whole warp
#pragma unroll
            for (int d = 0; d < N; ++d) {
                const unsigned b = __ballot_sync(FULL, s_cap[d * V + i] > 0);
                if (lane == 0) s_R[d * NR + rho] = b;
            }
            const unsigned bt = __ballot_sync(FULL, s_tcap[i] > 0);
            const unsigned be = __ballot_sync(FULL, s_exc[i] > 0);
            if (lane == 0) {
                s_T[rho] = bt;
                s_E[rho] = be;
            }
        }
    };
    // with only_round, just the cells whose row the last Augment round changed
    // (a boundary arc's residual changes only by a push of its own cell)
    auto rebuild_hm = [&](bool only_round) {
        for (int h = tid; h < C::HL; h += NT) {
            int lx, ly, lz, d;
            halo3_src<TY, TZ>(h, lx, ly, lz, d);
            const int rho = lz * TY + ly;
            if (only_round && s_dirty[rho] != 2) continue;
            const int i = rho * TX + lx;
            s_hm[h] = s_cap[d * V + i] > 0 ? s_hl[h] : INT_MAX;
        }
    };

    // ---- stage the tile --------------------------------------------------------
    const bool full = ox + TX <= g.X && oy + TY <= g.Y && oz + TZ <= g.Z;
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
        for (int c = tid; c < (N + 2) * NR; c += NT) {
            const int p = c / NR, rho = c % NR;
            const int *plane = p < N ? st.cap + (size_t)p * n : p == N ? st.tcap : st.exc;
            const size_t v0 = ((size_t)(oz + rho / TY) * g.Y + (oy + rho % TY)) * g.X + ox;
            bulk_g2s(s_cap + p * V + rho * TX, plane + v0, TX * 4, mbar);
        }
        for (int i4 = tid; i4 < V / 4; i4 += NT) *(int4 *)&s_lab[i4 * 4] = make_int4(0, 0, 0, 0);
    } else {
        for (int i = tid; i < V; i += NT) {
            const int lx = i % TX, rho = i / TX;
            const int x = ox + lx, y = oy + rho % TY, z = oz + rho / TY;
            const bool in = x < g.X && y < g.Y && z < g.Z;
            const size_t v = ((size_t)z * g.Y + y) * g.X + x;
#pragma unroll
            for (int d = 0; d < N; ++d) s_cap[d * V + i] = in ? st.cap[d * n + v] : 0;
            s_tcap[i] = in ? st.tcap[v] : 0;
            s_exc[i] = in ? st.exc[v] : 0;
            s_lab[i] = 0;
        }
    }
    for (int rho = tid; rho < NR; rho += NT) s_dirty[rho] = 0;
    for (int h = tid; h < C::HL; h += NT) {
        int lx, ly, lz, d;
        halo3_src<TY, TZ>(h, lx, ly, lz, d);
        const int x = ox + lx + arc_dx(6, d), y = oy + ly + arc_dy(6, d), z = oz + lz + arc_dz(6, d);
        const bool ing = x >= 0 && x < g.X && y >= 0 && y < g.Y && z >= 0 && z < g.Z;
        s_hl[h] = ing ? st.lab[((size_t)z * g.Y + y) * g.X + x] : dinf;
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
    rebuild_hm(false);
    __syncthreads();
    DIAG_LAP(0);

    // ---- graph-warp helpers (warp 0) ------------------------------------------
    auto next_stage = [&](int k) -> int {
        int best = INT_MAX;
        for (int h = lane; h < C::HL; h += 32) {
            const int v = s_hl[h];
            if (v < dinf && v + 1 > k && v + 1 < best) best = v + 1;
        }
        return __reduce_min_sync(FULL, best);
    };
    // seed rows of T_k: residual arc to t, or to a halo cell w with d(w) < k
    auto seed_rows = [&](int k, u32 (&sd)[RPL]) {
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int rho = lane * RPL + j;
            u32 s = 0u;
            if (lrow) {
                s = s_T[rho];
                if (s_hm[C::B_MX + rho] < k) s |= 1u;
                if (s_hm[C::B_PX + rho] < k) s |= 1u << (TX - 1);
            }
            sd[j] = s;
        }
        for (int z = 0; z < TZ; ++z) {
            const u32 bm = __ballot_sync(FULL, s_hm[C::B_MY + z * TX + lane] < k);
            const u32 bp = __ballot_sync(FULL, s_hm[C::B_PY + z * TX + lane] < k);
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                const int rho = lane * RPL + j;
                if (rho == z * TY) sd[j] |= bm;
                if (rho == z * TY + TY - 1) sd[j] |= bp;
            }
        }
        for (int y = 0; y < TY; ++y) {
            const u32 bm = __ballot_sync(FULL, s_hm[C::B_MZ + y * TX + lane] < k);
            const u32 bp = __ballot_sync(FULL, s_hm[C::B_PZ + y * TX + lane] < k);
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                const int rho = lane * RPL + j;
                if (rho == y) sd[j] |= bm;
                if (rho == (TZ - 1) * TY + y) sd[j] |= bp;
            }
        }
    };
    auto load_masks = [&](u32 (&Rm)[N][RPL]) {
#pragma unroll
        for (int j = 0; j < RPL; ++j)
#pragma unroll
            for (int d = 0; d < N; ++d) Rm[d][j] = lrow ? s_R[d * NR + lane * RPL + j] : 0u;
    };
    // one backward BFS step: vertices with a residual arc into f
    auto expand = [&](const u32 (&Rm)[N][RPL], const u32 (&f)[RPL], u32 (&out)[RPL]) {
        const u32 up = __shfl_up_sync(FULL, f[RPL - 1], 1);
        const u32 dn = __shfl_down_sync(FULL, f[0], 1);
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int rho = lane * RPL + j, y = rho % TY, z = rho / TY;
            const u32 zm = __shfl_up_sync(FULL, f[j], LZ);    // row rho - TY
            const u32 zp = __shfl_down_sync(FULL, f[j], LZ);  // row rho + TY
            const u32 fa = j == 0 ? up : f[j - 1];            // row rho - 1
            const u32 fb = j == RPL - 1 ? dn : f[j + 1];      // row rho + 1
            u32 a = (Rm[0][j] & (f[j] >> 1)) | (Rm[1][j] & (f[j] << 1));
            if (y < TY - 1) a |= Rm[2][j] & fb;
            if (y > 0) a |= Rm[3][j] & fa;
            if (z < TZ - 1) a |= Rm[4][j] & zp;
            if (z > 0) a |= Rm[5][j] & zm;
            out[j] = a;
        }
    };
    u32 Cl[RPL];
#pragma unroll
    for (int j = 0; j < RPL; ++j) Cl[j] = 0;
    auto flood = [&](const u32 (&sd)[RPL]) {
        u32 Rm[N][RPL], fr[RPL], inc[RPL];
        load_masks(Rm);
        bool any = false;
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const u32 f = row_fill32(sd[j] & ~Cl[j], Rm[0][j] & ~Cl[j], Rm[1][j] & ~Cl[j]);
            Cl[j] |= f;
            inc[j] = f;
            fr[j] = f;
            any |= f != 0u;
        }
        while (__any_sync(FULL, any)) {
            u32 nf[RPL];
            expand(Rm, fr, nf);
            any = false;
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                const u32 f = row_fill32(nf[j] & ~Cl[j], Rm[0][j] & ~Cl[j], Rm[1][j] & ~Cl[j]);
                Cl[j] |= f;
                inc[j] |= f;
                fr[j] = f;
                any |= f != 0u;
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
        for (int j = 0; j < RPL; ++j) m |= lrow && (Cl[j] & s_E[lane * RPL + j]) != 0u;
        return __any_sync(FULL, m);
    };
    auto write_labels = [&](int k) {
        for (int rho = warp; rho < NR; rho += NW)
            if ((s_inc[rho] >> lane) & 1u) s_lab[rho * TX + lane] = k;
    };

    const int klimit = sa.partial ? (sa.sweep_dev ? *sa.sweep_dev : sa.sweep) : INT_MAX;
    long long flow_acc = 0;
    int rounds = 0, stages = 0, epoch = 0;
    bool err = false, any_aug = false;
    bool cl_valid = true;

    // ---- ARD stages ------------------------------------------------------------
    for (int k = 0;;) {
        DIAG_MARK();
        if (warp == 0) {
            DIAG_ADD(2, 1);
            u32 sd[RPL];
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
                    u32 Rm[N][RPL], vis[RPL], fr[RPL], want[RPL];
                    load_masks(Rm);
                    seed_rows(k, fr);
                    int lmax = 0;
                    bool pending = false;
#pragma unroll
                    for (int j = 0; j < RPL; ++j) {
                        const int rho = lane * RPL + j;
                        const u32 ex = lrow ? s_E[rho] & Cl[j] : 0u;  // excess that can reach T_k lies in the closure
                        vis[j] = fr[j];
                        if (lrow) {
                            s_layer[1 * NR + rho] = fr[j];
                            s_vis[rho] = 0u;  // vertices that receive excess in this round's push
                        }
                        if (fr[j] & ex) lmax = 1;
                        want[j] = ex & ~vis[j];
                        pending |= want[j] != 0u;
                    }
                    int L = 1;
                    while (__any_sync(FULL, pending)) {
                        u32 nf[RPL];
                        expand(Rm, fr, nf);
                        bool any = false;
#pragma unroll
                        for (int j = 0; j < RPL; ++j) {
                            nf[j] &= ~vis[j];
                            any |= nf[j] != 0u;
                        }
                        if (!__any_sync(FULL, any)) break;
                        ++L;
                        pending = false;
#pragma unroll
                        for (int j = 0; j < RPL; ++j) {
                            const int rho = lane * RPL + j;
                            vis[j] |= nf[j];
                            fr[j] = nf[j];
                            if (L <= LCAP) {
                                if (lrow) s_layer[L * NR + rho] = nf[j];
                            } else {
                                const int tg = deep_tag3(epoch, L);
                                for (u32 m = nf[j]; m; m &= m - 1) s_lab[rho * TX + __ffs((int)m) - 1] = tg;
                            }
                            if (nf[j] & want[j]) lmax = L;
                            want[j] &= ~nf[j];
                            pending |= want[j] != 0u;
                        }
                    }
                    lmax = __reduce_max_sync(FULL, lmax);
                    if (lane == 0) s_ctl[2] = lmax;
                    DIAG_ADD(6, L);
                }
                __syncthreads();
                DIAG_LAP(4);
                const int Lmax = s_ctl[2];
                if (Lmax == 0) break;  // no excess vertex reaches T_k: stage done
                ++rounds;
                // layered push, top layer first: layer L pushes only to layer L-1
                // (to T_k from layer 1), so every arc has one writer per step.
                // Only vertices that had excess when the round began (s_E) or
                // received some in an earlier step of it (s_vis) can push, so
                // rows without such a vertex of layer L are passed over.
                u32 *s_recv = s_vis;
                for (int L = Lmax; L >= 1; --L) {
                    const int tgL = deep_tag3(epoch, L), tgL1 = deep_tag3(epoch, L - 1);
                    const bool lo_mask = L - 1 <= LCAP;
                    for (int rho = warp; rho < NR; rho += NW) {
                        const u32 P = (L <= LCAP ? s_layer[L * NR + rho] : FULL) & (s_E[rho] | s_recv[rho]);
                        if (!P) continue;
                        u32 A[N];
                        if (L > 1 && lo_mask) {
                            const u32 *lay = s_layer + (L - 1) * NR;
                            const u32 l0 = lay[rho];
                            A[0] = s_R[0 * NR + rho] & (l0 >> 1);
                            A[1] = s_R[1 * NR + rho] & (l0 << 1);
#pragma unroll
                            for (int d = 2; d < N; ++d) {
                                const int o = d == 2 ? 1 : d == 3 ? -1 : d == 4 ? TY : -TY;
                                A[d] = row_has(d, rho) ? (s_R[d * NR + rho] & lay[rho + o]) : 0u;
                            }
                        }
                        bool pushed = false;
                        const int lx = lane, i = rho * TX + lx;
                        const int ly = rho % TY, lz = rho / TY;
                        bool act = (P >> lx) & 1u;
                        if (act && L > LCAP) act = s_lab[i] == tgL;
                        int e = act ? s_exc[i] : 0;
                        if (e > 0) {
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
                                    const int nx = lx + arc_dx(6, d), ny = ly + arc_dy(6, d), nz = lz + arc_dz(6, d);
                                    if (nx >= 0 && nx < TX && ny >= 0 && ny < TY && nz >= 0 && nz < TZ) continue;
                                    const int c = s_cap[d * V + i];
                                    if (c > 0 && s_hl[halo3<TY, TZ>(d, lx, ly, lz)] < k) {
                                        const int dl = min(e, c);
                                        s_cap[d * V + i] = c - dl;
                                        e -= dl;
                                    }
                                }
                            } else {
#pragma unroll
                                for (int d = 0; d < N; ++d) {
                                    if (e == 0) break;
                                    const int nx = lx + arc_dx(6, d), ny = ly + arc_dy(6, d), nz = lz + arc_dz(6, d);
                                    bool adm;
                                    if (lo_mask) {
                                        adm = (A[d] >> lx) & 1u;
                                    } else {
                                        adm = nx >= 0 && nx < TX && ny >= 0 && ny < TY && nz >= 0 && nz < TZ &&
                                              s_lab[i + arc_off(d)] == tgL1 && s_cap[d * V + i] > 0;
                                    }
                                    if (!adm) continue;
                                    const int j = i + arc_off(d);
                                    const int c = s_cap[d * V + i];
                                    const int dl = min(e, c);
                                    s_cap[d * V + i] = c - dl;
                                    s_cap[(d ^ 1) * V + j] += dl;
                                    atomicAdd(&s_exc[j], dl);
                                    atomicOr(&s_recv[j >> 5], 1u << (j & 31));
                                    e -= dl;
                                }
                            }
                            s_exc[i] = e;
                            pushed = e != e0;
                        }
                        if (__any_sync(FULL, pushed) && lane < 5) {
                            const int o = lane == 0 ? -TY : lane == 1 ? -1 : lane == 2 ? 0 : lane == 3 ? 1 : TY;
                            const int rr = rho + o;
                            if (rr >= 0 && rr < NR) s_dirty[rr] = 2;  // changed in this round
                        }
                    }
                    __syncthreads();
                }
                DIAG_LAP(7);
                rebuild_masks(true);  // a push changes its row and the rows one step away in y and z only
                rebuild_hm(true);
                __syncthreads();
                for (int rho = tid; rho < NR; rho += NT)
                    if (s_dirty[rho] == 2) s_dirty[rho] = 1;
                DIAG_LAP(3);
                DIAG_ADD(8, Lmax);
            }
            if (warp == 0) cl_valid = false;  // the residual graph changed
        }
        if (kn == INT_MAX) break;
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
                u32 sd[RPL];
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
        const int lx = i % TX, rho = i / TX, ly = rho % TY, lz = rho / TY;
        const int x = ox + lx, y = oy + ly, z = oz + lz;
        if (!(x < g.X && y < g.Y && z < g.Z)) continue;
        const size_t v = ((size_t)z * g.Y + y) * g.X + x;
        const bool dirty = s_dirty[rho] != 0;
        bool perim = false;
#pragma unroll
        for (int d = 0; d < N; ++d) {
            const int nx = lx + arc_dx(6, d), ny = ly + arc_dy(6, d), nz = lz + arc_dz(6, d);
            const int gx = x + arc_dx(6, d), gy = y + arc_dy(6, d), gz = z + arc_dz(6, d);
            const bool intile = nx >= 0 && nx < TX && ny >= 0 && ny < TY && nz >= 0 && nz < TZ;
            const bool ing = gx >= 0 && gx < g.X && gy >= 0 && gy < g.Y && gz >= 0 && gz < g.Z;
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
        const int lab = ((s_vis[rho] >> lx) & 1u) ? s_lab[i] : dinf;
        if (perim) st.lab_next[v] = lab;
        else st.lab[v] = lab;
        if (s_exc[i] > 0 && lab < dinf) left = 1;
    }
    left = __syncthreads_or(left);
    unsigned long long f = (unsigned long long)flow_acc;
    for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(FULL, f, o);
    if (lane == 0 && f) atomicAdd(&s_flow, f);
    __syncthreads();
    if (tid == 0) {
        DIAG_LAP(10);
        DIAG_ADD(11, clock64() - diag_t0);
        DIAG_ADD(12, 1);
        DIAG_ADD(13, rounds);
        DIAG_FLUSH();
        if (s_flow) atomicAdd(st.flow_t, s_flow);
        st.disc[r] = 1;
        st.left_active[r] = (unsigned char)left;
        if (err) atomicExch(&st.ctr[kError], 1);
        atomicAdd(&sa.c64->stages, (unsigned long long)stages);
        atomicAdd(&sa.c64->rounds, (unsigned long long)rounds);
        atomicAdd(&sa.c64->discharges, 1ull);
        const unsigned long long live =
            (unsigned long long)min(TX, g.X - ox) * min(TY, g.Y - oy) * min(TZ, g.Z - oz);
        atomicAdd(&sa.c64->discharged_vertices, live);
    }
}

template <int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT, (Cfg3D<TY, TZ, NT>::MINB)) ard_discharge3d_kernel(const Geom g, const DevState st, const SweepArgs sa) {
    const int r = blockIdx.x;
    if (!st.active[r]) return;
    __shared__ __align__(8) unsigned long long s_mbar;
    if (threadIdx.x == 0) mbar_init(&s_mbar, 1);
    __syncthreads();
    unsigned phase = 0;
    discharge3d_region<TY, TZ, NT>(g, st, sa, r, &s_mbar, phase);
}

template <int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT, (Cfg3D<TY, TZ, NT>::MINB))
ard_discharge3d_batch_kernel(const Inst *__restrict__ insts, const int2 *__restrict__ items, const int *count,
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
        discharge3d_region<TY, TZ, NT>(I.g, I.st, a, w.y, &s_mbar, phase);
    }
}

template <int TY, int TZ, int NT>
static cudaError_t launch3d(const Geom &g, const DevState &st, const SweepArgs &sa, cudaStream_t s) {
    using C = Cfg3D<TY, TZ, NT>;
    auto k = ard_discharge3d_kernel<TY, TZ, NT>;
    {
        const cudaError_t e_at = ensure_smem_attr((const void *)k, (int)C::smem);
        if (e_at != cudaSuccess) return e_at;
    }
    k<<<g.nreg, NT, C::smem, s>>>(g, st, sa);
    return cudaGetLastError();
}

template <int TY, int TZ, int NT>
static cudaError_t launch3d_batch(const Inst *insts, const int2 *items, const int *count, int *head,
                                  const SweepArgs &sa, int blocks, cudaStream_t s) {
    using C = Cfg3D<TY, TZ, NT>;
    auto k = ard_discharge3d_batch_kernel<TY, TZ, NT>;
    {
        const cudaError_t e_at = ensure_smem_attr((const void *)k, (int)C::smem);
        if (e_at != cudaSuccess) return e_at;
    }
    // persistent blocks: at least as many as can be resident
    const int resident = device_sms() * C::MINB;
    k<<<blocks > resident ? blocks : resident, NT, C::smem, s>>>(insts, items, count, head, sa);
    return cudaGetLastError();
}

bool discharge3d_supported(int tx, int ty, int tz) {
    return tx == 32 && ((ty == 16 && tz == 8) || (ty == 8 && tz == 8) || (ty == 8 && tz == 4) || (ty == 4 && tz == 4) ||
                        (ty == 8 && tz == 2));
}

cudaError_t launch_discharge3d(const Geom &g, const DevState &st, const SweepArgs &sa, cudaStream_t stream) {
    if (g.tx == 32 && g.ty == 16 && g.tz == 8) return launch3d<16, 8, 512>(g, st, sa, stream);
    if (g.tx == 32 && g.ty == 8 && g.tz == 8) return launch3d<8, 8, 256>(g, st, sa, stream);
    if (g.tx == 32 && g.ty == 8 && g.tz == 4) return launch3d<8, 4, 256>(g, st, sa, stream);
    if (g.tx == 32 && g.ty == 4 && g.tz == 4) return launch3d<4, 4, 128>(g, st, sa, stream);
    if (g.tx == 32 && g.ty == 8 && g.tz == 2) return launch3d<8, 2, 128>(g, st, sa, stream);
    return cudaErrorInvalidValue;
}

cudaError_t launch_discharge3d_batch(int tx, int ty, int tz, const Inst *insts, const int2 *items, const int *count,
                                     int *head, const SweepArgs &sa, int blocks, cudaStream_t stream) {
    if (tx == 32 && ty == 16 && tz == 8) return launch3d_batch<16, 8, 512>(insts, items, count, head, sa, blocks, stream);
    if (tx == 32 && ty == 8 && tz == 8) return launch3d_batch<8, 8, 256>(insts, items, count, head, sa, blocks, stream);
    if (tx == 32 && ty == 8 && tz == 4) return launch3d_batch<8, 4, 256>(insts, items, count, head, sa, blocks, stream);
    if (tx == 32 && ty == 4 && tz == 4) return launch3d_batch<4, 4, 128>(insts, items, count, head, sa, blocks, stream);
    if (tx == 32 && ty == 8 && tz == 2) return launch3d_batch<8, 2, 128>(insts, items, count, head, sa, blocks, stream);
    return cudaErrorInvalidValue;
}

}  // namespace mf
