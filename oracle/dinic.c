/*
 * CPU oracle — TEST INFRASTRUCTURE ONLY.  Nothing in the solver library may
 * call, link or load this file; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg do.
 *
 * Maximum flow of the explicit s-t network of a grid instance, by Dinic's
 * algorithm (BFS level graph + blocking flow with current-arc pointers,
 * iterative, no recursion).  This is the plain definition of the problem the
 * paper solves (Sec. 2, Eq. 1 and the max-flow/min-cut duality stated with
 * it): vertices V = grid cells plus s and t, an arc s->v of capacity cs(v), an
 * arc v->t of capacity ct(v), and for every neighbour edge {u,w} the two arcs
 * u->w and w->u, both of capacity c(u,w) (the paper takes E symmetric).  No
 * terminal reduction, no regions, no labels: nothing of the region-discharge
 * method is used here.
 *
 * Outputs: the flow value |f| (int64), and the two canonical minimum cuts:
 *   S_min = vertices reachable from s in the residual network of the maximum
 *           flow (the minimal source set),
 *   S_max = grid vertices from which t is NOT reachable in that residual
 *           network (the cut (T-bar, T) of Sec. 2 with T = {v : v -> t}).
 *
 * Grid conventions (an interface, shared with the input generators): vertex
 * v = (z*Y + y)*X + x; nlink[h*n + v] is the capacity of the edge between v
 * and v + FWD[h], where FWD is the forward half-stencil below.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const int FWD4[2][3] = {{1, 0, 0}, {0, 1, 0}};
static const int FWD8[4][3] = {{1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {-1, 1, 0}};
static const int FWD6[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
/* Sec. 7.1: the displacements of the synthetic networks in the order listed,
 * read as (dx, dy), the first pair written (1,0), (0,1) as in FWD4;
 * connectivity c (code 100 + c) uses the first c/2 */
static const int FWDP[14][3] = {{1, 0, 0}, {0, 1, 0}, {1, 2, 0}, {2, 1, 0}, {1, 3, 0}, {3, 1, 0}, {2, 3, 0},
                                {3, 2, 0}, {0, 2, 0}, {2, 0, 0}, {2, 2, 0}, {3, 3, 0}, {3, 4, 0}, {4, 2, 0}};

/* forward half-stencil of a connectivity; returns H (number of half-dirs) */
int orc_stencil(int conn, const int (**fwd)[3]) {
    switch (conn) {
    case 4: *fwd = FWD4; return 2;
    case 8: *fwd = FWD8; return 4;
    case 6: *fwd = FWD6; return 3;
    default:
        if (conn >= 108 && conn <= 128 && conn % 4 == 0) { *fwd = FWDP; return (conn - 100) / 2; }
        *fwd = 0;
        return 0;
    }
}

typedef struct {
    int64_t nn;        /* nodes: n grid vertices + s + t */
    int64_t na;        /* arcs */
    int64_t *first;    /* [nn+1] CSR offsets */
    int64_t *head;     /* [na] */
    int64_t *rev;      /* [na] index of the paired reverse arc */
    int64_t *cap;      /* [na] residual capacity */
} net_t;

static void net_free(net_t *g) {
    free(g->first); free(g->head); free(g->rev); free(g->cap);
    memset(g, 0, sizeof(*g));
}

/* Build the explicit network.  Arc pairs (a, a^1 in the pair list) are laid
 * out into CSR by a counting sort on the tail. */
static int net_build(net_t *g, const int64_t dims[3], int conn, const int32_t *cs,
                     const int32_t *ct, const int32_t *nlink) {
    const int (*fwd)[3];
    int H = orc_stencil(conn, &fwd);
    int64_t X = dims[0], Y = dims[1], Z = dims[2], n = X * Y * Z;
    int64_t s = n, t = n + 1;
    memset(g, 0, sizeof(*g));
    if (H == 0) return -1;
    /* count pairs */
    int64_t np = 2 * n;
    for (int h = 0; h < H; ++h)
        for (int64_t z = 0; z < Z; ++z)
            for (int64_t y = 0; y < Y; ++y)
                for (int64_t x = 0; x < X; ++x) {
                    int64_t xx = x + fwd[h][0], yy = y + fwd[h][1], zz = z + fwd[h][2];
                    if (xx < 0 || xx >= X || yy < 0 || yy >= Y || zz < 0 || zz >= Z) continue;
                    ++np;
                }
    int64_t na = 2 * np;
    int64_t *ptail = malloc(sizeof(int64_t) * na), *phead = malloc(sizeof(int64_t) * na);
    int64_t *pcap = malloc(sizeof(int64_t) * na);
    if (!ptail || !phead || !pcap) { free(ptail); free(phead); free(pcap); return -2; }
    int64_t k = 0;
    for (int64_t v = 0; v < n; ++v) {
        ptail[k] = s; phead[k] = v; pcap[k] = cs[v]; ++k;   /* s -> v */
        ptail[k] = v; phead[k] = s; pcap[k] = 0; ++k;       /* reverse */
        ptail[k] = v; phead[k] = t; pcap[k] = ct[v]; ++k;   /* v -> t */
        ptail[k] = t; phead[k] = v; pcap[k] = 0; ++k;       /* reverse */
    }
    for (int h = 0; h < H; ++h)
        for (int64_t z = 0; z < Z; ++z)
            for (int64_t y = 0; y < Y; ++y)
                for (int64_t x = 0; x < X; ++x) {
                    int64_t xx = x + fwd[h][0], yy = y + fwd[h][1], zz = z + fwd[h][2];
                    if (xx < 0 || xx >= X || yy < 0 || yy >= Y || zz < 0 || zz >= Z) continue;
                    int64_t v = (z * Y + y) * X + x, w = (zz * Y + yy) * X + xx;
                    int64_t c = nlink[(int64_t)h * n + v];
                    ptail[k] = v; phead[k] = w; pcap[k] = c; ++k;
                    ptail[k] = w; phead[k] = v; pcap[k] = c; ++k;
                }
    g->nn = n + 2;
    g->na = na;
    g->first = calloc(g->nn + 1, sizeof(int64_t));
    g->head = malloc(sizeof(int64_t) * na);
    g->rev = malloc(sizeof(int64_t) * na);
    g->cap = malloc(sizeof(int64_t) * na);
    int64_t *pos = malloc(sizeof(int64_t) * na);
    int64_t *fill = malloc(sizeof(int64_t) * (g->nn + 1));
    if (!g->first || !g->head || !g->rev || !g->cap || !pos || !fill) {
        free(ptail); free(phead); free(pcap); free(pos); free(fill); net_free(g); return -2;
    }
    for (int64_t a = 0; a < na; ++a) g->first[ptail[a] + 1]++;
    for (int64_t u = 0; u < g->nn; ++u) g->first[u + 1] += g->first[u];
    memcpy(fill, g->first, sizeof(int64_t) * (g->nn + 1));
    for (int64_t a = 0; a < na; ++a) pos[a] = fill[ptail[a]]++;
    for (int64_t a = 0; a < na; ++a) {
        int64_t p = pos[a];
        g->head[p] = phead[a];
        g->cap[p] = pcap[a];
        g->rev[p] = pos[a ^ 1];
    }
    free(ptail); free(phead); free(pcap); free(pos); free(fill);
    return 0;
}

/* BFS level graph from s over arcs of positive residual capacity. */
static int bfs_levels(const net_t *g, int64_t s, int64_t t, int64_t *level, int64_t *queue) {
    for (int64_t u = 0; u < g->nn; ++u) level[u] = -1;
    int64_t qh = 0, qt = 0;
    level[s] = 0;
    queue[qt++] = s;
    while (qh < qt) {
        int64_t u = queue[qh++];
        for (int64_t a = g->first[u]; a < g->first[u + 1]; ++a) {
            int64_t w = g->head[a];
            if (g->cap[a] > 0 && level[w] < 0) {
                level[w] = level[u] + 1;
                queue[qt++] = w;
            }
        }
    }
    return level[t] >= 0;
}

/* One blocking flow on the level graph (iterative DFS with current arcs). */
static int64_t blocking_flow(net_t *g, int64_t s, int64_t t, int64_t *level, int64_t *cur,
                             int64_t *path, int64_t *nodes) {
    int64_t total = 0;
    for (int64_t u = 0; u < g->nn; ++u) cur[u] = g->first[u];
    int64_t depth = 0;
    int64_t u = s;
    nodes[0] = s;
    for (;;) {
        if (u == t) {
            int64_t delta = INT64_MAX;
            for (int64_t i = 0; i < depth; ++i)
                if (g->cap[path[i]] < delta) delta = g->cap[path[i]];
            int64_t cut = -1;
            for (int64_t i = 0; i < depth; ++i) {
                g->cap[path[i]] -= delta;
                g->cap[g->rev[path[i]]] += delta;
                if (cut < 0 && g->cap[path[i]] == 0) cut = i;
            }
            total += delta;
            depth = cut;        /* retreat to the tail of the first saturated arc */
            u = nodes[depth];
            continue;
        }
        int64_t a = cur[u];
        while (a < g->first[u + 1] &&
               !(g->cap[a] > 0 && level[g->head[a]] == level[u] + 1))
            ++a;
        cur[u] = a;
        if (a < g->first[u + 1]) {
            path[depth] = a;
            u = g->head[a];
            nodes[++depth] = u;
        } else {
            level[u] = -1;      /* dead end: remove u from the level graph */
            if (depth == 0) break;
            --depth;
            u = nodes[depth];
            cur[u]++;
        }
    }
    return total;
}

/*
 * Maximum flow value of the grid instance; fills smin/smax (n bytes each, 1 =
 * source side) when non-null and the number of Dinic phases when non-null.
 * Returns -1 on bad arguments, -2 on allocation failure.
 */
int64_t orc_maxflow(const int64_t dims[3], int conn, const int32_t *cs, const int32_t *ct,
                    const int32_t *nlink, uint8_t *smin, uint8_t *smax, int64_t *phases_out) {
    net_t g;
    int rc = net_build(&g, dims, conn, cs, ct, nlink);
    if (rc) return rc;
    int64_t n = dims[0] * dims[1] * dims[2], s = n, t = n + 1;
    int64_t *level = malloc(sizeof(int64_t) * g.nn), *queue = malloc(sizeof(int64_t) * g.nn);
    int64_t *cur = malloc(sizeof(int64_t) * g.nn);
    int64_t *path = malloc(sizeof(int64_t) * (g.nn + 1)), *nodes = malloc(sizeof(int64_t) * (g.nn + 1));
    if (!level || !queue || !cur || !path || !nodes) {
        free(level); free(queue); free(cur); free(path); free(nodes); net_free(&g); return -2;
    }
    int64_t flow = 0, phases = 0;
    while (bfs_levels(&g, s, t, level, queue)) {
        flow += blocking_flow(&g, s, t, level, cur, path, nodes);
        ++phases;
    }
    if (smin) {
        /* residual reachability from s */
        bfs_levels(&g, s, t, level, queue);
        for (int64_t v = 0; v < n; ++v) smin[v] = level[v] >= 0;
    }
    if (smax) {
        /* vertices that reach t: reverse BFS from t; x reaches t if an arc
         * x->y of positive residual capacity leads to a vertex y that does */
        for (int64_t u = 0; u < g.nn; ++u) level[u] = -1;
        int64_t qh = 0, qt = 0;
        level[t] = 0;
        queue[qt++] = t;
        while (qh < qt) {
            int64_t y = queue[qh++];
            for (int64_t a = g.first[y]; a < g.first[y + 1]; ++a) {
                int64_t x = g.head[a];
                if (g.cap[g.rev[a]] > 0 && level[x] < 0) {
                    level[x] = 0;
                    queue[qt++] = x;
                }
            }
        }
        for (int64_t v = 0; v < n; ++v) smax[v] = level[v] < 0;
    }
    if (phases_out) *phases_out = phases;
    free(level); free(queue); free(cur); free(path); free(nodes);
    net_free(&g);
    return flow;
}

/*
 * Same maximum flow, exported as a maximum PREFLOW in the solver's residual
 * layout (see verify.c): res[d*n+v] residual of the arc v -> v + D(d),
 * tres[v] residual of v -> t, exc[v] = residual of s -> v.  Saturating the
 * unused part of every s-link turns the maximum flow into a maximum preflow
 * whose excess sits exactly where s still reaches (Sec. 2, Init saturates all
 * s-links).  Returns the flow value (or < 0 on failure).
 */
int64_t orc_maxflow_state(const int64_t dims[3], int conn, const int32_t *cs, const int32_t *ct,
                          const int32_t *nlink, int32_t *res, int32_t *tres, int32_t *exc) {
    net_t g;
    int rc = net_build(&g, dims, conn, cs, ct, nlink);
    if (rc) return rc;
    const int (*fwd)[3];
    int H = orc_stencil(conn, &fwd);
    int64_t n = dims[0] * dims[1] * dims[2], s = n, t = n + 1;
    int64_t *level = malloc(sizeof(int64_t) * g.nn), *queue = malloc(sizeof(int64_t) * g.nn);
    int64_t *cur = malloc(sizeof(int64_t) * g.nn);
    int64_t *path = malloc(sizeof(int64_t) * (g.nn + 1)), *nodes = malloc(sizeof(int64_t) * (g.nn + 1));
    if (!level || !queue || !cur || !path || !nodes) {
        free(level); free(queue); free(cur); free(path); free(nodes); net_free(&g); return -2;
    }
    int64_t flow = 0;
    while (bfs_levels(&g, s, t, level, queue))
        flow += blocking_flow(&g, s, t, level, cur, path, nodes);
    memset(res, 0, sizeof(int32_t) * 2 * H * n);
    for (int64_t v = 0; v < n; ++v) {
        int64_t x = v % dims[0], y = (v / dims[0]) % dims[1], z = v / (dims[0] * dims[1]);
        for (int64_t a = g.first[v]; a < g.first[v + 1]; ++a) {
            int64_t w = g.head[a];
            if (w == t) { tres[v] = (int32_t)g.cap[a]; continue; }
            if (w == s) continue;
            int64_t wx = w % dims[0], wy = (w / dims[0]) % dims[1], wz = w / (dims[0] * dims[1]);
            for (int d = 0; d < 2 * H; ++d) {
                int sg = (d & 1) ? -1 : 1;
                if (wx == x + sg * fwd[d >> 1][0] && wy == y + sg * fwd[d >> 1][1] &&
                    wz == z + sg * fwd[d >> 1][2]) {
                    res[(int64_t)d * n + v] = (int32_t)g.cap[a];
                    break;
                }
            }
        }
    }
    for (int64_t a = g.first[s]; a < g.first[s + 1]; ++a) exc[g.head[a]] = (int32_t)g.cap[a];
    free(level); free(queue); free(cur); free(path); free(nodes);
    net_free(&g);
    return flow;
}
