/*
 * A plain C99 client of include/mf.h: reads one grid instance from a binary
 * file, solves it through the C ABI and writes the flow value and both
 * minimum cuts.  The tests use it to check that the boundary works from C
 * without the Python binding.
 *
 * input file (little-endian):  int32 ndim, conn, X, Y, Z; int32 tile[3];
 *                              int32 cs[n]; int32 ct[n]; int32 nlink[conn/2][n]
 * output file:                 int64 flow; int32 sweeps; uint8 smin[n]; uint8 smax[n]
 * exit status: 0 on success, 1 on bad usage or I/O, 2 + mf_status on a
 * failing call (the message goes to stderr).
 *
 * usage: mf_solve_file IN OUT
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "mf.h"

static int fail_call(const char *what, mf_status s, const mf_grid *g) {
    fprintf(stderr, "%s failed (%d): %s\n", what, (int)s, mf_last_error(g));
    return 2 + (int)s;
}

static int read_i32(FILE *f, int32_t *p, size_t count) { return fread(p, 4, count, f) == count; }

int main(int argc, char **argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s IN OUT\n", argv[0]);
        return 1;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 1;
    int32_t hdr[8];
    if (!read_i32(in, hdr, 8)) return 1;
    const int ndim = hdr[0], conn = hdr[1];
    const int64_t dims[3] = {hdr[2], hdr[3], hdr[4]};
    const int32_t tile[3] = {hdr[5], hdr[6], hdr[7]};
    const size_t n = (size_t)dims[0] * (size_t)dims[1] * (size_t)dims[2];
    const size_t H = (size_t)conn / 2;
    int32_t *cs = malloc(n * 4), *ct = malloc(n * 4), *nl = malloc(H * n * 4);
    uint8_t *smin = malloc(n), *smax = malloc(n);
    if (!cs || !ct || !nl || !smin || !smax) return 1;
    if (!read_i32(in, cs, n) || !read_i32(in, ct, n) || !read_i32(in, nl, H * n)) return 1;
    fclose(in);

    mf_grid *g = NULL;
    mf_status s = mf_create_grid(&g, ndim, dims, conn, tile, NULL);
    if (s != MF_OK) return fail_call("mf_create_grid", s, NULL);
    /* out-of-order calls are reported, not fatal */
    if (mf_solve(g, NULL, NULL) != MF_ESTATE) {
        fprintf(stderr, "mf_solve before mf_set_caps did not report MF_ESTATE\n");
        return 1;
    }
    s = mf_set_caps(g, cs, ct, nl, 0);
    if (s != MF_OK) return fail_call("mf_set_caps", s, g);
    mf_opts opts;
    mf_default_opts(&opts);
    mf_stats stats;
    s = mf_solve(g, &opts, &stats);
    if (s != MF_OK) return fail_call("mf_solve", s, g);
    int64_t flow = 0;
    s = mf_flow_value(g, &flow);
    if (s != MF_OK) return fail_call("mf_flow_value", s, g);
    s = mf_get_cut(g, smin, 0, 0);
    if (s == MF_OK) s = mf_get_cut(g, smax, 1, 0);
    if (s != MF_OK) return fail_call("mf_get_cut", s, g);
    mf_destroy(g);

    FILE *out = fopen(argv[2], "wb");
    if (!out) return 1;
    const int32_t sweeps = stats.sweeps;
    if (fwrite(&flow, 8, 1, out) != 1 || fwrite(&sweeps, 4, 1, out) != 1 || fwrite(smin, 1, n, out) != n ||
        fwrite(smax, 1, n, out) != n)
        return 1;
    fclose(out);
    printf("flow %lld sweeps %d\n", (long long)flow, (int)sweeps);
    free(cs);
    free(ct);
    free(nl);
    free(smin);
    free(smax);
    return 0;
}
