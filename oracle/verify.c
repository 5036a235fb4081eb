/*
 * CPU oracle — TEST INFRASTRUCTURE ONLY (see dinic.c).
 *
 * Independent checker of a claimed maximum preflow on a grid instance.  It
 * follows the definitions of Sec. 2 directly:
 *   - capacity and antisymmetry constraints: with residual capacities
 *     r(u,w) = c(u,w) - f(u,w) and r(w,u) = c(w,u) + f(u,w) on a symmetric
 *     edge, 0 <= r and r(u,w) + r(w,u) = 2 c(u,w);
 *   - every s-link saturated (the Init procedure of Sec. 2), the sink link
 *     residual r(v,t) in [0, ct(v)];
 *   - preflow constraint: the excess recomputed from the residuals,
 *     e(v) = cs(v) - f(v,t) - sum_w f(v,w), is >= 0 and equals the claimed one;
 *   - flow value |f| = sum_v f(v,t);
 *   - maximality (Sec. 2): {v : e(v) > 0} does not reach t in G_f;
 *   - the cut cost of Eq. 1 on the ORIGINAL capacities equals |f| for
 *     S_min = closure of {e > 0} under residual arcs and for
 *     S_max = complement of {v : v -> t in G_f}; a cut of cost |f| next to a
 *     feasible preflow of value |f| certifies both optimal (weak duality).
 *
 * Residual layout read here (the solver's export format): res[d*n + v] is the
 * residual capacity of the arc from v to v + D(d), with D(2h) = +FWD[h] and
 * D(2h+1) = -FWD[h]; tres[v] is the residual of v->t; exc[v] the excess.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int orc_stencil(int conn, const int (**fwd)[3]);

/* neighbour of v along arc direction d, or -1 outside the grid */
static int64_t nbr(const int64_t dims[3], const int (*fwd)[3], int64_t x, int64_t y, int64_t z, int d) {
    int sg = (d & 1) ? -1 : 1;
    int64_t xx = x + sg * fwd[d >> 1][0], yy = y + sg * fwd[d >> 1][1], zz = z + sg * fwd[d >> 1][2];
    if (xx < 0 || xx >= dims[0] || yy < 0 || yy >= dims[1] || zz < 0 || zz >= dims[2]) return -1;
    return (zz * dims[1] + yy) * dims[0] + xx;
}

/* capacity of the edge carried by arc direction d at v (its neighbour w) */
static int64_t edge_cap(const int64_t dims[3], int H, const int32_t *nlink, int64_t v, int64_t w, int d) {
    int64_t n = dims[0] * dims[1] * dims[2];
    (void)H;
    return (d & 1) ? nlink[(int64_t)(d >> 1) * n + w] : nlink[(int64_t)(d >> 1) * n + v];
}

/*
 * Cut cost of Eq. 1 for source set S (S[v] = 1: v on the source side):
 *   sum_{v not in S} cs(v) + sum_{v in S} ct(v) + sum_{u in S, w not in S} c(u,w).
 */
int64_t orc_cut_cost(const int64_t dims[3], int conn, const int32_t *cs, const int32_t *ct,
                     const int32_t *nlink, const uint8_t *S) {
    const int (*fwd)[3];
    int H = orc_stencil(conn, &fwd);
    int64_t n = dims[0] * dims[1] * dims[2], cost = 0;
    for (int64_t v = 0; v < n; ++v) cost += S[v] ? ct[v] : cs[v];
    for (int64_t z = 0; z < dims[2]; ++z)
        for (int64_t y = 0; y < dims[1]; ++y)
            for (int64_t x = 0; x < dims[0]; ++x) {
                int64_t v = (z * dims[1] + y) * dims[0] + x;
                for (int h = 0; h < H; ++h) {
                    int64_t w = nbr(dims, fwd, x, y, z, 2 * h);
                    if (w < 0) continue;
                    if (S[v] != S[w]) cost += nlink[(int64_t)h * n + v];
                }
            }
    return cost;
}

/*
 * Forward closure (dir = 0): in[v] = 1 for seeds; adds every w reachable by
 * arcs of positive residual.  Backward closure (dir = 1): adds every u that
 * has a residual arc into the set.  Plain FIFO BFS.
 */
void orc_closure(const int64_t dims[3], int conn, const int32_t *res, int dir, uint8_t *set) {
    const int (*fwd)[3];
    int H = orc_stencil(conn, &fwd);
    int N = 2 * H;
    int64_t n = dims[0] * dims[1] * dims[2];
    int64_t *q = malloc(sizeof(int64_t) * (n ? n : 1));
    int64_t qh = 0, qt = 0;
    for (int64_t v = 0; v < n; ++v) if (set[v]) q[qt++] = v;
    while (qh < qt) {
        int64_t v = q[qh++];
        int64_t x = v % dims[0], y = (v / dims[0]) % dims[1], z = v / (dims[0] * dims[1]);
        for (int d = 0; d < N; ++d) {
            int64_t w = nbr(dims, fwd, x, y, z, d);
            if (w < 0 || set[w]) continue;
            /* forward: arc v->w; backward: arc w->v, i.e. direction d^1 at w */
            int32_t r = dir == 0 ? res[(int64_t)d * n + v] : res[(int64_t)(d ^ 1) * n + w];
            if (r > 0) { set[w] = 1; q[qt++] = w; }
        }
    }
    free(q);
}

#define FAIL(...) do { if (msg) snprintf(msg, msglen, __VA_ARGS__); rc = __LINE__; goto done; } while (0)

/*
 * Returns 0 when every check passes, otherwise a nonzero code and a message.
 * smin_claim / smax_claim may be null (not compared).  out[0..3] receive
 * |f| recomputed, |S_min|, |S_max| and the cut cost of S_min.
 */
int orc_verify(const int64_t dims[3], int conn, const int32_t *cs, const int32_t *ct,
               const int32_t *nlink, const int32_t *res, const int32_t *tres, const int32_t *exc,
               int64_t flow_claim, const uint8_t *smin_claim, const uint8_t *smax_claim,
               char *msg, int msglen, int64_t *out) {
    const int (*fwd)[3];
    int H = orc_stencil(conn, &fwd);
    int N = 2 * H;
    int64_t n = dims[0] * dims[1] * dims[2];
    int rc = 0;
    uint8_t *smin = calloc(n ? n : 1, 1), *tset = calloc(n ? n : 1, 1);
    if (msg && msglen) msg[0] = 0;
    if (H == 0) FAIL("bad connectivity %d", conn);
    int64_t flow = 0;
    for (int64_t z = 0; z < dims[2]; ++z)
        for (int64_t y = 0; y < dims[1]; ++y)
            for (int64_t x = 0; x < dims[0]; ++x) {
                int64_t v = (z * dims[1] + y) * dims[0] + x;
                if (tres[v] < 0 || tres[v] > ct[v])
                    FAIL("sink residual out of range at v=%lld: %d (ct=%d)", (long long)v, tres[v], ct[v]);
                int64_t fvt = (int64_t)ct[v] - tres[v];
                flow += fvt;
                int64_t e = (int64_t)cs[v] - fvt;
                for (int d = 0; d < N; ++d) {
                    int64_t w = nbr(dims, fwd, x, y, z, d);
                    int32_t r = res[(int64_t)d * n + v];
                    if (w < 0) {
                        if (r != 0) FAIL("arc leaving the grid has residual %d at v=%lld d=%d", r, (long long)v, d);
                        continue;
                    }
                    int64_t c = edge_cap(dims, H, nlink, v, w, d);
                    int32_t rb = res[(int64_t)(d ^ 1) * n + w];
                    if (r < 0 || rb < 0) FAIL("negative residual at v=%lld d=%d", (long long)v, d);
                    if ((int64_t)r + rb != 2 * c)
                        FAIL("antisymmetry broken at v=%lld d=%d: %d + %d != 2*%lld", (long long)v, d, r, rb, (long long)c);
                    e -= c - r;     /* f(v,w) = c - r(v,w) */
                }
                if (e < 0) FAIL("negative excess %lld at v=%lld", (long long)e, (long long)v);
                if (e != exc[v]) FAIL("excess mismatch at v=%lld: recomputed %lld, claimed %d", (long long)v, (long long)e, exc[v]);
            }
    if (flow != flow_claim) FAIL("flow value mismatch: recomputed %lld, claimed %lld", (long long)flow, (long long)flow_claim);
    for (int64_t v = 0; v < n; ++v) smin[v] = exc[v] > 0;
    orc_closure(dims, conn, res, 0, smin);
    for (int64_t v = 0; v < n; ++v)
        if (smin[v] && tres[v] > 0) FAIL("not maximal: v=%lld reached from an excess vertex has sink residual %d", (long long)v, tres[v]);
    for (int64_t v = 0; v < n; ++v) tset[v] = tres[v] > 0;
    orc_closure(dims, conn, res, 1, tset);
    for (int64_t v = 0; v < n; ++v) tset[v] = !tset[v];  /* S_max */
    int64_t cmin = orc_cut_cost(dims, conn, cs, ct, nlink, smin);
    int64_t cmax = orc_cut_cost(dims, conn, cs, ct, nlink, tset);
    if (cmin != flow) FAIL("cut cost of S_min %lld != flow %lld", (long long)cmin, (long long)flow);
    if (cmax != flow) FAIL("cut cost of S_max %lld != flow %lld", (long long)cmax, (long long)flow);
    int64_t nmin = 0, nmax = 0;
    for (int64_t v = 0; v < n; ++v) {
        nmin += smin[v]; nmax += tset[v];
        if (smin[v] && !tset[v]) FAIL("S_min not inside S_max at v=%lld", (long long)v);
        if (smin_claim && (smin_claim[v] != 0) != smin[v]) FAIL("claimed S_min differs at v=%lld", (long long)v);
        if (smax_claim && (smax_claim[v] != 0) != tset[v]) FAIL("claimed S_max differs at v=%lld", (long long)v);
    }
    if (out) { out[0] = flow; out[1] = nmin; out[2] = nmax; out[3] = cmin; }
done:
    free(smin); free(tset);
    return rc;
}
