// Region discharge of P-ARD: one thread block discharges one region (a grid
// tile) per sweep, entirely in shared memory.
//
// What one block computes is Procedure ARD of Sec. 4.2 on the region network
// G^R of Sec. 3: vertices R plus the boundary B^R (the halo of the tile) plus
// s, t; arcs inside R, arcs R -> B^R with their residual capacity, arcs into
// t; the arcs B^R -> R carry capacity 0 and are never loaded.
//
//   for each stage k in {0} U {d(w)+1 : w in B^R, d(w) < d_inf} (ascending;
//   with partial discharges only k <= sweep, Sec. 6.2):
//       Augment(R, T_k),  T_k = {t} U {w in B^R : d(w) < k}
//   region-relabel: d(u) = min{k : u -> T_k}, else d_inf  (Sec. 4.2, the
//   ARD variant of the region-relabel of Sec. 5.1)
//
// Augment(R, T_k) (Procedure Augment) is done in synchronous rounds.  A round
// is a backward BFS from T_k over residual arcs inside R, giving every vertex
// its residual distance dist to T_k, followed by one pass over the BFS
// layers from the highest to 1 in which every vertex with excess pushes
// min(excess, residual) along arcs to the next lower layer (to t or to
// boundary vertices of T_k from layer 1).  Every push starts at a vertex with
// excess and ends at a vertex that reached T_k in the round's BFS; these two
// properties are what the proofs of Statement 3 and Corollaries 1-2 (Sec. 4.2)
// need from the augmentations, so the order-free parallel pushes keep ARD's
// guarantees (a push into a vertex that reaches T_k adds a reverse arc whose
// tail already reaches T_a for every a >= k; a push out of an excess vertex
// adds a reverse arc inside the set reachable from the excess).  A stage ends
// when no vertex with excess reaches T_k, exactly the loop condition of
// Procedure Augment.  Paths through boundary vertices are not followed: by
// Corollary 1 a boundary vertex w with d(w) >= k cannot reach T_k.
#pragma once

#include <climits>

#include "mf_internal.cuh"

namespace mf {

template <int CONN, int TX, int TY, int TZ, int NT>
struct TileCfg {
    static constexpr int N = arcs_of(CONN);        // arcs per vertex
    static constexpr bool D3 = (CONN == 6);
    static constexpr int R = radius_of(CONN);      // halo width: the longest displacement
    static constexpr int V = TX * TY * TZ;         // vertices per tile
    static constexpr int PX = TX + 2 * R, PY = TY + 2 * R, PZ = D3 ? TZ + 2 * R : 1;
    static constexpr int P = PX * PY * PZ;         // padded tile (halo ring)
    static constexpr int VPT = (V + NT - 1) / NT;  // vertices per thread
    static constexpr size_t smem = (size_t)(N + 3) * V * sizeof(int) + (size_t)P * sizeof(int);
};

// block-wide max / min of an int with triple-buffered shared slots (one barrier)
__device__ __forceinline__ int block_reduce_max(int v, int *slots, int &ph) {
    int *s = slots + ph;
    ph = ph == 2 ? 0 : ph + 1;
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) atomicMax(s, v);
    if (threadIdx.x == 0) slots[ph] = INT_MIN;
    __syncthreads();
    return *s;
}

template <int CONN, int TX, int TY, int TZ, int NT>
__device__ __forceinline__ void discharge_region(const Geom &g, const DevState &st, const SweepArgs &sa,
                                                 const int r) {
    using C = TileCfg<CONN, TX, TY, TZ, NT>;
    constexpr int N = C::N, V = C::V, VPT = C::VPT;
    extern __shared__ __align__(16) int smem[];
    int *s_cap = smem;              // [N][V] residual of arc i -> i + D(d)
    int *s_tcap = s_cap + N * V;    // [V]
    int *s_exc = s_tcap + V;        // [V]
    int *s_dist = s_exc + V;        // [V] BFS distance / region label
    int *s_hlab = s_dist + V;       // [P] labels of B^R (d_inf elsewhere)
    __shared__ int s_red[3];
    __shared__ unsigned long long s_flow;

    const int tid = threadIdx.x;
    if (tid < 3) s_red[tid] = INT_MIN;
    if (tid == 0) s_flow = 0;
    int ph = 0;

    const int rx = r % g.RX, ry = (r / g.RX) % g.RY, rz = r / (g.RX * g.RY);
    const int ox = rx * TX, oy = ry * TY, oz = rz * TZ;
    const size_t n = (size_t)g.n;
    const int dinf = g.dinf;

    // ---- stage the tile (planes of R) and the labels of B^R ---------------
    for (int i = tid; i < V; i += NT) {
        const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
        const int x = ox + lx, y = oy + ly, z = oz + lz;
        const bool in = x < g.X && y < g.Y && z < g.Z;
        const size_t v = ((size_t)z * g.Y + y) * g.X + x;
#pragma unroll
        for (int d = 0; d < N; ++d) s_cap[d * V + i] = in ? st.cap[d * n + v] : 0;
        s_tcap[i] = in ? st.tcap[v] : 0;
        s_exc[i] = in ? st.exc[v] : 0;
    }
    for (int p = tid; p < C::P; p += NT) {
        const int px = p % C::PX, py = (p / C::PX) % C::PY, pz = p / (C::PX * C::PY);
        const int lx = px - C::R, ly = py - C::R, lz = C::D3 ? pz - C::R : 0;
        const bool out = lx < 0 || lx >= TX || ly < 0 || ly >= TY || lz < 0 || lz >= TZ;
        // cells outside the tile that are the head of some stencil arc from it
        bool adj = false;
#pragma unroll
        for (int d = 0; d < C::N; ++d) {
            const int sx = lx - arc_dx(CONN, d), sy = ly - arc_dy(CONN, d), sz = lz - arc_dz(CONN, d);
            adj |= sx >= 0 && sx < TX && sy >= 0 && sy < TY && sz >= 0 && sz < TZ;
        }
        adj &= out;
        const int x = ox + lx, y = oy + ly, z = oz + lz;
        const bool ing = x >= 0 && x < g.X && y >= 0 && y < g.Y && z >= 0 && z < g.Z;
        s_hlab[p] = (adj && ing) ? st.lab[((size_t)z * g.Y + y) * g.X + x] : dinf;
    }

    // per-thread vertex geometry: in-tile arcs and arcs to in-grid boundary vertices
    int my_i[VPT];
    unsigned in_m[VPT], halo_m[VPT];
    int hbase[VPT];
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        const int i = tid + q * NT;
        my_i[q] = i;
        in_m[q] = 0;
        halo_m[q] = 0;
        hbase[q] = 0;
        if (i >= V) continue;
        const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
        const int x = ox + lx, y = oy + ly, z = oz + lz;
        if (!(x < g.X && y < g.Y && z < g.Z)) continue;  // ragged tile: no vertex here
        hbase[q] = ((lz + (C::D3 ? C::R : 0)) * C::PY + (ly + C::R)) * C::PX + (lx + C::R);
#pragma unroll
        for (int d = 0; d < N; ++d) {
            const int dx = arc_dx(CONN, d), dy = arc_dy(CONN, d), dz = arc_dz(CONN, d);
            const int nlx = lx + dx, nly = ly + dy, nlz = lz + dz;
            const bool intile = nlx >= 0 && nlx < TX && nly >= 0 && nly < TY && nlz >= 0 && nlz < TZ;
            const int gx = x + dx, gy = y + dy, gz = z + dz;
            const bool ing = gx >= 0 && gx < g.X && gy >= 0 && gy < g.Y && gz >= 0 && gz < g.Z;
            if (intile) in_m[q] |= 1u << d;
            else if (ing) halo_m[q] |= 1u << d;
        }
    }
    __syncthreads();

    auto ioff = [](int d) { return arc_dx(CONN, d) + arc_dy(CONN, d) * TX + arc_dz(CONN, d) * TX * TY; };
    auto hoff = [](int d) { return arc_dx(CONN, d) + arc_dy(CONN, d) * C::PX + arc_dz(CONN, d) * C::PX * C::PY; };

    // next stage value above k: min{d(w)+1 > k : w in B^R, d(w) < d_inf}
    auto next_stage = [&](int k) {
        int best = INT_MAX;
        for (int p = tid; p < C::P; p += NT) {
            const int h = s_hlab[p];
            if (h < dinf && h + 1 > k && h + 1 < best) best = h + 1;
        }
        return -block_reduce_max(-best, s_red, ph);  // best <= INT_MAX, so -best > INT_MIN
    };

    const int klimit = sa.partial ? (sa.sweep_dev ? *sa.sweep_dev : sa.sweep) : INT_MAX;
    long long flow_acc = 0;
    int rounds = 0, stages = 0;
    bool err = false;
    const bool prd = sa.variant == 2;

    // ---- Procedure PRD (Sec. 3): push-relabel inside R ------------------------
    // Rounds of an exact relabel (the region-relabel of Sec. 5.1 with unit
    // arc lengths: dist(u) = 1 if u -> t, else the least d(w) + 1 over the
    // residual arcs into boundary vertices w, and dist(v) + 1 over residual
    // arcs inside R; the largest labels that stay valid given d on B^R, so
    // never below the current ones) followed by pushes along admissible arcs
    // (dist(u) = dist(v) + 1) from the highest excess layer down, until no
    // vertex of R with excess has a label below d_inf.
    if (prd) {
        ++stages;
        for (int round = 0;; ++round) {
            if (round >= sa.max_rounds) { err = true; break; }
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                const int i = my_i[q];
                if (i >= V) continue;
                int dv = s_tcap[i] > 0 ? 1 : kInf;
#pragma unroll
                for (int d = 0; d < N; ++d)
                    if ((halo_m[q] >> d & 1u) && s_cap[d * V + i] > 0) {
                        const int h = s_hlab[hbase[q] + hoff(d)];
                        if (h < dinf && h + 1 < dv) dv = h + 1;
                    }
                s_dist[i] = dv;
            }
            __syncthreads();
            for (;;) {  // relax to the fixed point (values only fall; a stale read only delays)
                int ch = 0;
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    const int i = my_i[q];
                    if (i >= V) continue;
                    int dv = s_dist[i];
#pragma unroll
                    for (int d = 0; d < N; ++d) {
                        if (!(in_m[q] >> d & 1u) || s_cap[d * V + i] <= 0) continue;
                        const int dj = s_dist[i + ioff(d)];
                        if (dj != kInf && dj + 1 < dv) dv = dj + 1;
                    }
                    if (dv < s_dist[i]) {
                        s_dist[i] = dv;
                        ch = 1;
                    }
                }
                if (!__syncthreads_or(ch)) break;
            }
            int lm = 0;
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                const int i = my_i[q];
                if (i < V && s_exc[i] > 0 && s_dist[i] < dinf && s_dist[i] > lm) lm = s_dist[i];
            }
            int Lc = block_reduce_max(lm, s_red, ph);
            if (Lc == 0) break;  // no active vertex left in R
            ++rounds;
            while (Lc >= 1) {
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    const int i = my_i[q];
                    if (i >= V || s_dist[i] != Lc) continue;
                    int e = s_exc[i];
                    if (e <= 0) continue;
                    if (Lc == 1 && s_tcap[i] > 0) {
                        const int dl = min(e, s_tcap[i]);
                        s_tcap[i] -= dl;
                        e -= dl;
                        flow_acc += dl;
                    }
#pragma unroll
                    for (int d = 0; d < N; ++d) {
                        if (e == 0) break;
                        const int c = s_cap[d * V + i];
                        if (c <= 0) continue;
                        if (halo_m[q] >> d & 1u) {  // out of the region, to a boundary vertex one label lower
                            if (s_hlab[hbase[q] + hoff(d)] + 1 != Lc) continue;
                            const int dl = min(e, c);
                            s_cap[d * V + i] = c - dl;
                            e -= dl;
                        } else if (in_m[q] >> d & 1u) {
                            const int j = i + ioff(d);
                            if (s_dist[j] != Lc - 1) continue;
                            const int dl = min(e, c);
                            s_cap[d * V + i] = c - dl;
                            s_cap[(d ^ 1) * V + j] += dl;
                            atomicAdd(&s_exc[j], dl);
                            e -= dl;
                        }
                    }
                    s_exc[i] = e;
                }
                __syncthreads();
                // the next lower layer that holds excess
                int nx = 0;
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    const int i = my_i[q];
                    if (i < V && s_exc[i] > 0 && s_dist[i] < Lc && s_dist[i] > nx) nx = s_dist[i];
                }
                Lc = block_reduce_max(nx, s_red, ph);
            }
        }
    }

    // ---- Augment(R, T_k) for every stage ------------------------------------
    for (int k = 0; !prd;) {
        if (k > klimit) break;
        ++stages;
        for (int round = 0;; ++round) {
            if (round >= sa.max_rounds) { err = true; break; }
            // BFS layer 1: vertices with a residual arc into T_k
            int unl = 0;
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                const int i = my_i[q];
                if (i >= V) continue;
                bool seed = s_tcap[i] > 0;
#pragma unroll
                for (int d = 0; d < N; ++d)
                    if (!seed && (halo_m[q] >> d & 1u) && s_cap[d * V + i] > 0 && s_hlab[hbase[q] + hoff(d)] < k)
                        seed = true;
                s_dist[i] = seed ? 1 : kInf;
                if (!seed && s_exc[i] > 0) unl = 1;
            }
            int L = 1;
            if (__syncthreads_or(unl)) {
                for (;;) {
                    int newly = 0;
                    unl = 0;
#pragma unroll
                    for (int q = 0; q < VPT; ++q) {
                        const int i = my_i[q];
                        if (i >= V || s_dist[i] != kInf) continue;
#pragma unroll
                        for (int d = 0; d < N; ++d) {
                            if ((in_m[q] >> d & 1u) && s_cap[d * V + i] > 0 && s_dist[i + ioff(d)] == L) {
                                s_dist[i] = L + 1;
                                newly = 1;
                                break;
                            }
                        }
                        if (s_dist[i] == kInf && s_exc[i] > 0) unl = 1;
                    }
                    const int any_new = __syncthreads_or(newly);
                    const int any_unl = __syncthreads_or(unl);
                    ++L;
                    if (!any_new || !any_unl) break;
                }
            }
            // highest layer holding excess that reaches T_k
            int lm = 0;
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                const int i = my_i[q];
                if (i < V && s_exc[i] > 0 && s_dist[i] != kInf && s_dist[i] > lm) lm = s_dist[i];
            }
            const int Lmax = block_reduce_max(lm, s_red, ph);
            if (Lmax == 0) break;  // no excess vertex reaches T_k: stage done
            ++rounds;
            // layered push, top layer first; a vertex at layer L only pushes to
            // layer L-1, so every arc has one writer per step
            for (int Lc = Lmax; Lc >= 1; --Lc) {
#pragma unroll
                for (int q = 0; q < VPT; ++q) {
                    const int i = my_i[q];
                    if (i >= V || s_dist[i] != Lc) continue;
                    int e = s_exc[i];
                    if (e <= 0) continue;
                    if (Lc == 1) {
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
                            if (!(halo_m[q] >> d & 1u)) continue;
                            const int c = s_cap[d * V + i];
                            if (c > 0 && s_hlab[hbase[q] + hoff(d)] < k) {
                                const int dl = min(e, c);
                                s_cap[d * V + i] = c - dl;
                                e -= dl;
                            }
                        }
                    } else {
#pragma unroll
                        for (int d = 0; d < N; ++d) {
                            if (e == 0) break;
                            if (!(in_m[q] >> d & 1u)) continue;
                            const int j = i + ioff(d);
                            const int c = s_cap[d * V + i];
                            if (c > 0 && s_dist[j] == Lc - 1) {
                                const int dl = min(e, c);
                                s_cap[d * V + i] = c - dl;
                                s_cap[(d ^ 1) * V + j] += dl;
                                atomicAdd(&s_exc[j], dl);
                                e -= dl;
                            }
                        }
                    }
                    s_exc[i] = e;
                }
                __syncthreads();
            }
        }
        if (err) break;
        const int kn = next_stage(k);
        if (kn == INT_MAX) break;
        k = kn;
    }

    // ---- region-relabel: d(u) = min{k : u -> T_k}, else d_inf ----------------
    // (PRD keeps the exact unit-length labels of its last round)
    auto flood = [&](int k) {
        for (;;) {
            int ch = 0;
#pragma unroll
            for (int q = 0; q < VPT; ++q) {
                const int i = my_i[q];
                if (i >= V || s_dist[i] != kInf) continue;
#pragma unroll
                for (int d = 0; d < N; ++d) {
                    if ((in_m[q] >> d & 1u) && s_cap[d * V + i] > 0 && s_dist[i + ioff(d)] <= k) {
                        s_dist[i] = k;
                        ch = 1;
                        break;
                    }
                }
            }
            if (!__syncthreads_or(ch)) break;
        }
    };
    if (!prd) {
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        const int i = my_i[q];
        if (i < V) s_dist[i] = s_tcap[i] > 0 ? 0 : kInf;
    }
    __syncthreads();
    flood(0);
    }
    for (int k = 0; !prd;) {
        const int kn = next_stage(k);
        if (kn == INT_MAX) break;
        k = kn;
#pragma unroll
        for (int q = 0; q < VPT; ++q) {
            const int i = my_i[q];
            if (i >= V || s_dist[i] != kInf) continue;
#pragma unroll
            for (int d = 0; d < N; ++d)
                if ((halo_m[q] >> d & 1u) && s_cap[d * V + i] > 0 && s_hlab[hbase[q] + hoff(d)] < k) {
                    s_dist[i] = k;
                    break;
                }
        }
        __syncthreads();
        flood(k);
    }

    // ---- write back ------------------------------------------------------------
    int left = 0;
#pragma unroll
    for (int q = 0; q < VPT; ++q) {
        const int i = my_i[q];
        if (i >= V) continue;
        const int lx = i % TX, ly = (i / TX) % TY, lz = i / (TX * TY);
        const int x = ox + lx, y = oy + ly, z = oz + lz;
        if (!(x < g.X && y < g.Y && z < g.Z)) continue;
        const size_t v = ((size_t)z * g.Y + y) * g.X + x;
#pragma unroll
        for (int d = 0; d < N; ++d) {
            const int c = s_cap[d * V + i];
            if (halo_m[q] >> d & 1u) {
                st.bout[d * n + v] = st.cap[d * n + v] - c;  // flow pushed across the boundary
                st.cap[d * n + v] = c;
            } else if (in_m[q] >> d & 1u) {
                st.cap[d * n + v] = c;
            }
        }
        st.tcap[v] = s_tcap[i];
        st.exc[v] = s_exc[i];
        const int lab = s_dist[i] >= dinf ? dinf : s_dist[i];
        if (halo_m[q]) st.lab_next[v] = lab;  // boundary vertex: fused after the sweep
        else st.lab[v] = lab;
        if (s_exc[i] > 0 && lab < dinf) left = 1;
    }
    left = __syncthreads_or(left);
    // flow into t of this discharge
    unsigned long long f = (unsigned long long)flow_acc;
    for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
    if ((tid & 31) == 0 && f) atomicAdd(&s_flow, f);
    __syncthreads();
    if (tid == 0) {
        if (s_flow) atomicAdd(st.flow_t, s_flow);
        st.disc[r] = 1;
        st.left_active[r] = (unsigned char)left;
        if (err) atomicExch(&st.ctr[kError], 1);
        atomicAdd(&sa.c64->stages, (unsigned long long)stages);
        atomicAdd(&sa.c64->rounds, (unsigned long long)rounds);
        atomicAdd(&sa.c64->discharges, 1ull);
        const unsigned long long live = (unsigned long long)min(TX, g.X - ox) * min(TY, g.Y - oy) * min(TZ, g.Z - oz);
        atomicAdd(&sa.c64->discharged_vertices, live);
    }
}

template <int CONN, int TX, int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT, 1) ard_discharge_kernel(const Geom g, const DevState st, const SweepArgs sa) {
    const int r = blockIdx.x;
    if (!st.active[r]) return;  // regions without active vertices are skipped (Sec. 5.3)
    discharge_region<CONN, TX, TY, TZ, NT>(g, st, sa, r);
}

// persistent blocks over a work queue of (instance, region) items of a batch
template <int CONN, int TX, int TY, int TZ, int NT>
__global__ void __launch_bounds__(NT, 1)
ard_discharge_batch_kernel(const Inst *__restrict__ insts, const int2 *__restrict__ items, const int *count,
                           int *head, const SweepArgs sa) {
    __shared__ int s_it;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_it = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_it;
        if (it >= *count) break;
        const int2 w = items[it];
        const Inst &I = insts[w.x];
        SweepArgs a = sa;
        a.c64 = I.c64;
        discharge_region<CONN, TX, TY, TZ, NT>(I.g, I.st, a, w.y);
    }
}

template <int CONN, int TX, int TY, int TZ, int NT>
static cudaError_t launch_batch_one(const Inst *insts, const int2 *items, const int *count, int *head,
                                    const SweepArgs &sa, int blocks, cudaStream_t s) {
    using C = TileCfg<CONN, TX, TY, TZ, NT>;
    auto k = ard_discharge_batch_kernel<CONN, TX, TY, TZ, NT>;
    {
        const cudaError_t e_at = ensure_smem_attr((const void *)k, (int)C::smem);
        if (e_at != cudaSuccess) return e_at;
    }
    k<<<blocks, NT, C::smem, s>>>(insts, items, count, head, sa);
    return cudaGetLastError();
}

// ---- instantiation table ----------------------------------------------------
template <int CONN, int TX, int TY, int TZ, int NT>
static cudaError_t launch_one(const Geom &g, const DevState &st, const SweepArgs &sa, cudaStream_t s) {
    using C = TileCfg<CONN, TX, TY, TZ, NT>;
    auto k = ard_discharge_kernel<CONN, TX, TY, TZ, NT>;
    {
        const cudaError_t e_at = ensure_smem_attr((const void *)k, (int)C::smem);
        if (e_at != cudaSuccess) return e_at;
    }
    k<<<g.nreg, NT, C::smem, s>>>(g, st, sa);
    return cudaGetLastError();
}

}  // namespace mf
