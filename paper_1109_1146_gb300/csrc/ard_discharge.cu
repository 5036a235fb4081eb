// Dispatch of the generic region discharge (ard_generic.cuh) over the tile
// shapes it is instantiated for, single grids and batches; the 2D and 3D
// bit-parallel kernels take the tiles they support, and the synthetic
// stencils of Sec. 7.1 are instantiated in ard_discharge_paper.cu.
#include "ard_generic.cuh"

namespace mf {

#define MF_TILES(X)                 \
    X(4, 64, 64, 1, 1024)           \
    X(8, 64, 64, 1, 1024)           \
    X(4, 32, 32, 1, 256)            \
    X(8, 32, 32, 1, 256)            \
    X(4, 64, 32, 1, 256)            \
    X(8, 64, 32, 1, 256)            \
    X(4, 32, 16, 1, 128)            \
    X(8, 32, 16, 1, 128)            \
    X(6, 16, 16, 16, 1024)          \
    X(6, 8, 8, 8, 256)              \
    X(6, 32, 16, 8, 1024)           \
    X(6, 32, 8, 8, 256)             \
    X(6, 32, 8, 4, 256)             \
    X(6, 32, 4, 4, 128)             \
    X(6, 32, 8, 2, 128)

bool discharge_supported(int conn, int tx, int ty, int tz) {
#define X(c, a, b, z, t) if (conn == c && tx == a && ty == b && tz == z) return true;
    MF_TILES(X)
#undef X
    return discharge_paper_supported(conn, tx, ty, tz);
}

size_t discharge_smem_bytes(int conn, int tx, int ty, int tz) {
#define X(c, a, b, z, t) if (conn == c && tx == a && ty == b && tz == z) return TileCfg<c, a, b, z, t>::smem;
    MF_TILES(X)
#undef X
    return discharge_paper_smem_bytes(conn, tx, ty, tz);
}

cudaError_t launch_discharge_batch(int conn, int tx, int ty, int tz, int variant, const Inst *insts,
                                   const int2 *items, const int *count, int *head, const SweepArgs &sa,
                                   int blocks, cudaStream_t stream) {
    if (variant == 0 && tz == 1 && discharge2d_supported(conn, tx, ty))
        return launch_discharge2d_batch(conn, tx, ty, insts, items, count, head, sa, blocks, stream);
    if (variant == 0 && conn == 6 && discharge3d_supported(tx, ty, tz))
        return launch_discharge3d_batch(tx, ty, tz, insts, items, count, head, sa, blocks, stream);
#define X(c, a, b, z, t) \
    if (conn == c && tx == a && ty == b && tz == z) return launch_batch_one<c, a, b, z, t>(insts, items, count, head, sa, blocks, stream);
    MF_TILES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_discharge(int conn, const Geom &g, const DevState &st, const SweepArgs &sa,
                             cudaStream_t stream) {
    if (sa.variant == 0 && g.tz == 1 && discharge2d_supported(conn, g.tx, g.ty))
        return launch_discharge2d(conn, g, st, sa, stream);
    if (sa.variant == 0 && conn == 6 && discharge3d_supported(g.tx, g.ty, g.tz))
        return launch_discharge3d(g, st, sa, stream);
#define X(c, a, b, z, t) \
    if (conn == c && g.tx == a && g.ty == b && g.tz == z) return launch_one<c, a, b, z, t>(g, st, sa, stream);
    MF_TILES(X)
#undef X
    if (is_paper(conn)) return launch_discharge_paper(conn, g, st, sa, stream);
    return cudaErrorInvalidValue;
}

}  // namespace mf
