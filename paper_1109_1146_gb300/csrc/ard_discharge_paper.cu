// The generic region discharge (ard_generic.cuh) for the synthetic networks
// of Sec. 7.1 (connectivity codes 100 + c, c = 8 .. 28; displacements up to
// 4): 32x32 tiles, and 64x32 / 64x64 at connectivity 8 (the paper's default,
// for the dependence on the number of regions); single solves.  A translation unit of its own, since the
// 28-arc instantiations are the slowest code of the library to compile.
#include "ard_generic.cuh"

namespace mf {

// the synthetic stencils of Sec. 7.1 (codes 100 + connectivity): single
// solves on 32x32 tiles, generic kernel only
#define MF_PAPER_TILES(X)           \
    X(108, 32, 32, 1, 256)          \
    X(112, 32, 32, 1, 256)          \
    X(116, 32, 32, 1, 256)          \
    X(120, 32, 32, 1, 256)          \
    X(124, 32, 32, 1, 256)          \
    X(128, 32, 32, 1, 256)          \
    X(108, 64, 32, 1, 256)          \
    X(108, 64, 64, 1, 1024)

bool discharge_paper_supported(int conn, int tx, int ty, int tz) {
#define X(c, a, b, z, t) if (conn == c && tx == a && ty == b && tz == z) return true;
    MF_PAPER_TILES(X)
#undef X
    return false;
}

size_t discharge_paper_smem_bytes(int conn, int tx, int ty, int tz) {
#define X(c, a, b, z, t) if (conn == c && tx == a && ty == b && tz == z) return TileCfg<c, a, b, z, t>::smem;
    MF_PAPER_TILES(X)
#undef X
    return 0;
}

cudaError_t launch_discharge_paper(int conn, const Geom &g, const DevState &st, const SweepArgs &sa,
                                   cudaStream_t stream) {
#define X(c, a, b, z, t) \
    if (conn == c && g.tx == a && g.ty == b && g.tz == z) return launch_one<c, a, b, z, t>(g, st, sa, stream);
    MF_PAPER_TILES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace mf
