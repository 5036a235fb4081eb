// Internal declarations of the P-ARD grid solver (not part of the C ABI).
//
// Device state, all int32 SoA planes over the full grid (plane[d][v], v =
// (z*Y + y)*X + x):
//   cap[d]   residual capacity of the arc v -> v + D(d) (Sec. 2, c_f);
//   tcap     residual capacity of v -> t;
//   exc      excess e_f(v);
//   lab      labeling d of Sec. 4.1 (values 0..d_inf);
//   lab_next new labels of region-boundary vertices written by a discharge and
//            committed by the fusion kernel (Algorithm 2 fuses labels after
//            all regions are discharged);
//   bout[d]  flow a discharge pushed across the region boundary on the arc
//            v -> v + D(d) (only entries of boundary arcs are used).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace mf {

constexpr int kInf = 0x7fffffff;   // "no distance" inside a discharge
constexpr int kHistBins = 16384;   // exact gap histogram bins; labels >= this share one bin

// The synthetic networks of Sec. 7.1 join every node to the nodes at the
// displacements of a fixed list; connectivity c takes its first c/2 entries.
// As forward half-stencil (dx, dy) in the list's order, except that the first
// pair is swapped to (1,0), (0,1) so that c = 4 is the 4-connected grid.
// Such a grid has the connectivity code 100 + c (c = 8, 12, ..., 28).
__host__ __device__ constexpr bool is_paper(int conn) { return conn > 100; }
__host__ __device__ constexpr int arcs_of(int conn) { return conn > 100 ? conn - 100 : conn; }
__host__ __device__ constexpr int paper_dx(int h) {
    return h == 0 ? 1 : h == 1 ? 0 : h == 2 ? 1 : h == 3 ? 2 : h == 4 ? 1 : h == 5 ? 3 : h == 6 ? 2 : h == 7 ? 3
         : h == 8 ? 0 : h == 9 ? 2 : h == 10 ? 2 : h == 11 ? 3 : h == 12 ? 3 : 4;
}
__host__ __device__ constexpr int paper_dy(int h) {
    return h == 0 ? 0 : h == 1 ? 1 : h == 2 ? 2 : h == 3 ? 1 : h == 4 ? 3 : h == 5 ? 1 : h == 6 ? 3 : h == 7 ? 2
         : h == 8 ? 2 : h == 9 ? 0 : h == 10 ? 2 : h == 11 ? 3 : h == 12 ? 4 : 2;
}
// largest |dx|, |dy| of a stencil (the width of the band of boundary vertices)
__host__ __device__ constexpr int radius_of(int conn) {
    return !is_paper(conn) ? 1 : arcs_of(conn) <= 4 ? 1 : arcs_of(conn) <= 8 ? 2 : arcs_of(conn) <= 24 ? 3 : 4;
}

// forward half-stencil and arc directions (see include/mf.h)
__host__ __device__ constexpr int fwd_dx(int conn, int h) {
    return is_paper(conn) ? paper_dx(h) : conn == 8 ? (h == 0 ? 1 : h == 1 ? 0 : h == 2 ? 1 : -1) : (h == 0 ? 1 : 0);
}
__host__ __device__ constexpr int fwd_dy(int conn, int h) {
    return is_paper(conn) ? paper_dy(h) : conn == 6 ? (h == 1 ? 1 : 0) : (h == 0 ? 0 : 1);
}
__host__ __device__ constexpr int fwd_dz(int conn, int h) { return (conn == 6 && h == 2) ? 1 : 0; }
__host__ __device__ constexpr int arc_dx(int conn, int d) { return (d & 1) ? -fwd_dx(conn, d >> 1) : fwd_dx(conn, d >> 1); }
__host__ __device__ constexpr int arc_dy(int conn, int d) { return (d & 1) ? -fwd_dy(conn, d >> 1) : fwd_dy(conn, d >> 1); }
__host__ __device__ constexpr int arc_dz(int conn, int d) { return (d & 1) ? -fwd_dz(conn, d >> 1) : fwd_dz(conn, d >> 1); }

struct Geom {
    int X, Y, Z;        // grid dims
    long long n;        // X*Y*Z
    int tx, ty, tz;     // tile (region) shape (powers of two)
    int sx, sy, sz;     // log2 of the tile shape
    int RX, RY, RZ;     // regions per axis
    int nreg;
    int dinf;           // d_inf = max(|B|, 1)  (Sec. 4.1)
};

struct DevState {
    int *cap, *tcap, *exc, *lab, *lab_next, *bout;
    unsigned char *active;       // [nreg] region has active vertices -> discharge next sweep
    unsigned char *disc;         // [nreg] region was discharged in the current sweep
    unsigned char *left_active;  // [nreg] a discharge left an active vertex (partial discharges)
    unsigned long long *flow_t;  // flow pushed into t by all discharges
    long long *flow0;            // sum of min(cs, ct) (terminal reduction)
    int *hist;                   // [kHistBins + 1] labels of boundary vertices
    int *ctr;                    // small counters, see Ctr
    int host;                    // nonzero: the planes live in host (Grace) memory, read over NVLink-C2C
};

// indices into DevState::ctr
enum Ctr : int {
    kActiveRegions = 0,  // regions active for the next sweep
    kError = 1,          // nonzero: a device loop hit its cap (MF_EROUNDLIMIT)
    kGap = 2,            // gap level g found this sweep (0 = none)
    kChanged = 3,        // cut extraction: a pass changed the set
    kStages = 4,         // ARD stages (low 32 bits; also kept in 64-bit below)
    kDischarges = 5,
    kGlrFlags = 8,       // 3 words: global relabel "grew" flags
    kGlrLevels = 11,     // global relabel: levels run
    kCtrWords = 16
};
struct Counters64 {
    unsigned long long stages, rounds, discharges, discharged_vertices;
};

struct SweepArgs {
    int sweep;          // 0-based sweep index
    const int *sweep_dev;  // if set, the sweep index is read here (sweeps inside a CUDA graph)
    int partial;        // partial discharges (Sec. 6.2)
    int max_rounds;     // Augment round cap per stage
    int variant;        // 0: bit-parallel 2D kernel where available, 1: generic kernel
    Counters64 *c64;
};

// ---- bulk asynchronous copies (TMA engine, no tensor map) into shared memory
// A transaction barrier (mbarrier) in shared memory counts the bytes of the
// copies issued against it; the phase completes when they have all landed.
// Addresses and sizes must be multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// one arrival that also announces the bytes the phase waits for
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// bounded wait for a phase: false if it did not complete within the limit
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned phase) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

// global -> shared bulk copy of `bytes` completing on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// order this thread's earlier generic-proxy accesses of shared memory before
// later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Optional phase probes (clock64 deltas and counters per discharge phase),
// compiled only with -DMF_DIAG; they expand to nothing otherwise.
#ifdef MF_DIAG
#define DIAG_DECL unsigned long long dg_[16] = {0}; long long dt_ = clock64();
#define DIAG_MARK() (dt_ = clock64())
#define DIAG_LAP(slot) do { const long long t_ = clock64(); dg_[slot] += t_ - dt_; dt_ = t_; } while (0)
#define DIAG_ADD(slot, v) (dg_[slot] += (unsigned long long)(v))
#define DIAG_FLUSH() do { for (int s_ = 0; s_ < 16; ++s_) if (dg_[s_]) atomicAdd(&mf_diag[s_], dg_[s_]); } while (0)
#else
#define DIAG_DECL
#define DIAG_MARK() ((void)0)
#define DIAG_LAP(slot) ((void)0)
#define DIAG_ADD(slot, v) ((void)0)
#define DIAG_FLUSH() ((void)0)
#endif

// one instance of a batch: its geometry, device state and statistics counters
struct Inst {
    Geom g;
    DevState st;
    Counters64 *c64;
    int conn;   // stencil of the instance (batched fusion kernels are per connectivity)
    int *h_ctr;      // device view of the pinned mirror of st.ctr
    void *h_fin;     // device view of the pinned record of the finished solve
};

// reduction.cu: region reduction of Sec. 8 (class codes per vertex)
constexpr unsigned char kStrongSource = 1, kStrongSink = 2, kWeakSource = 4, kWeakSink = 8;
constexpr int kRedMaxSmem = 232000;  // shared memory of one region network (tile plus a one-cell ring)
struct RedGeom {
    int X, Y, Z;        // grid dims
    int tx, ty, tz;     // region shape of the reduction
    int RX, RY, RZ;     // regions per axis
    int EX, EY, EZ, E;  // tile plus ring (EZ = 1 in 2D), cells
};
size_t reduction_smem_bytes(int conn, const RedGeom &rg);
bool reduction_supported(int conn, const int tile[3], RedGeom *out, const Geom &g);
// codes[v] for every vertex; counts[4] += strong sources, strong sinks, weak
// sources, weak sinks; *err = 1 if an Augment hit max_rounds
cudaError_t launch_region_reduction(int conn, const RedGeom &rg, const int *cs, const int *ct, const int *nl,
                                    unsigned char *codes, unsigned long long *counts, int max_rounds, int *err,
                                    cudaStream_t s);
cudaError_t launch_reduction_apply(int conn, const Geom &g, const unsigned char *codes, const int *cs, const int *ct,
                                   const int *nl, int *cs2, int *ct2, int *nl2, unsigned long long *konst,
                                   unsigned long long *konst2, cudaStream_t s);
cudaError_t launch_reduction_cut(size_t n, const unsigned char *codes, unsigned char *smin, unsigned char *smax,
                                 cudaStream_t s);

// batched global relabel (cut2d.cu for 2D grids, glr3d.cu for 3D grids with
// 32-wide tiles): one grid of a batch; the launcher fills the derived fields
struct GlrJob2 {
    Geom g;
    DevState st;
    int conn;                        // 4 or 8 (2D); 6 with ty/tz variants (3D)
    void *scratch;                   // the grid's cut scratch (masks and two level sets)
    int W64, BY, unit0;              // derived: row words, 64-row blocks, first work unit
    unsigned long long *M, *A, *B;   // derived: masks, level sets / closure sets
    unsigned char *smin, *smax;      // batched cut: the byte outputs
    int *hout;                       // device view of pinned host ints that receive the level
                                     // count (relabel: [0]) or the closure passes (cut: [0], [1]); or NULL
};
// device tables of a batched relabel, grown as needed and reused
struct GlrBatchBufs {
    void *jobs = nullptr, *units = nullptr, *chunks = nullptr, *rows = nullptr;
    size_t jobs_cap = 0, units_cap = 0, chunks_cap = 0, rows_cap = 0;
    int *any = nullptr;
    cudaError_t reserve(size_t jobs_bytes, size_t units_bytes, size_t chunks_bytes);
    // (job, row chunk) units of the batched mask builds, uploaded on stream s
    cudaError_t upload_rows(const std::vector<int2> &units, cudaStream_t s);
    ~GlrBatchBufs();
};
constexpr int kMaskRows = 16;  // grid rows per unit of a batched mask build
// the relabel of every listed 2D grid (tiles 32 or 64 wide), enqueued without
// waiting; each grid's levels land in its st.ctr[kGlrLevels]
cudaError_t glr2d_batch(const std::vector<GlrJob2> &jobs, GlrBatchBufs &bb, cudaStream_t s);
cudaError_t glr3d_batch(const std::vector<GlrJob2> &jobs, GlrBatchBufs &bb, cudaStream_t s);
// both cut closures of every listed grid (2D; 3D with 32-wide tiles) and the
// S_min / S_max bytes; the passes of each closure land in the job's hout
cudaError_t cut2d_batch(const std::vector<GlrJob2> &jobs, GlrBatchBufs &bb, cudaStream_t s);
cudaError_t cut3d_batch(const std::vector<GlrJob2> &jobs, GlrBatchBufs &bb, cudaStream_t s);
// one launch: hout[slot] = st.ctr[kGlrLevels] for every job of the uploaded
// table that has an hout
cudaError_t glr_batch_out(const GlrJob2 *jobs_dev, int njobs, int slot, cudaStream_t s);

// devinfo.cu: per-device launch facts, cached per (kernel, device)
int device_sms();  // SMs of the current device (1 if it cannot be queried)
// co-resident blocks of a cooperative kernel on the current device
cudaError_t coop_max_blocks(const void *kernel, int threads, size_t smem, int *out);
// allow `bytes` of dynamic shared memory for the kernel on the current device
cudaError_t ensure_smem_attr(const void *kernel, int bytes);

// launchers (ard_discharge.cu)
size_t discharge_smem_bytes(int conn, int tx, int ty, int tz);
bool discharge_supported(int conn, int tx, int ty, int tz);
// the synthetic stencils of Sec. 7.1 (codes 100 + c), generic kernel, single solves;
// their exact region-distance relabel (glr_stencil.cu, 32x32 tiles)
bool stencil_glr_supported(int conn, const Geom &g);
size_t stencil_glr_scratch_bytes(const Geom &g);
cudaError_t stencil_glr(int conn, const Geom &g, const DevState &st, void *scratch, cudaStream_t s);
bool discharge_paper_supported(int conn, int tx, int ty, int tz);
size_t discharge_paper_smem_bytes(int conn, int tx, int ty, int tz);
cudaError_t launch_discharge_paper(int conn, const Geom &g, const DevState &st, const SweepArgs &sa,
                                   cudaStream_t stream);
cudaError_t launch_discharge(int conn, const Geom &g, const DevState &st, const SweepArgs &sa,
                             cudaStream_t stream);
// cut2d.cu: residual closures S_min / S_max of a 2D grid on bit masks
size_t cut2d_scratch_bytes(const Geom &g, int conn);
// h_passes: NULL or pinned host int[2] that receives the passes of each
// closure asynchronously (valid after the stream is synchronised); no wait
cudaError_t cut2d(int conn, const Geom &g, const DevState &st, void *scratch, unsigned char *smin,
                  unsigned char *smax, int *h_passes, cudaStream_t s);
// message returned by mf_last_error(NULL) for calls without a handle (mf_capi.cu)
void set_static_error(const std::string &m);
// global relabel: exact region distance on bit masks (2D, tiles 32 or 64 wide)
bool glr2d_supported(const Geom &g);
// glr3d.cu: the same relabel for 3D 6-connected grids with 32-wide tiles
bool glr3d_supported(const Geom &g);
size_t glr3d_scratch_bytes(const Geom &g);
// the relabels enqueue everything without waiting; the number of BFS levels
// run is left in st.ctr[kGlrLevels]
cudaError_t glr3d(const Geom &g, const DevState &st, void *scratch, cudaStream_t s);
// both cut closures on bit masks (scratch: glr3d_scratch_bytes); passes += passes made
cudaError_t cut3d(const Geom &g, const DevState &st, void *scratch, unsigned char *smin, unsigned char *smax,
                  int *h_passes, cudaStream_t s);
cudaError_t glr2d(int conn, const Geom &g, const DevState &st, void *scratch, cudaStream_t s);
// persistent discharge over a work queue of (instance, region) items of one
// kernel type (connectivity, tile); blocks pull items until *count is reached
cudaError_t launch_discharge_batch(int conn, int tx, int ty, int tz, int variant, const Inst *insts,
                                   const int2 *items, const int *count, int *head, const SweepArgs &sa,
                                   int blocks, cudaStream_t stream);
// warm.cu: learned warm start (features, targets, projection to a preflow)
cudaError_t launch_warm_features(int conn, const Geom &g, const int *cs, const int *ct, const int *nl, float *x,
                                 cudaStream_t s);
cudaError_t launch_warm_targets(int conn, const Geom &g, const DevState &st, const int *cs, const int *ct,
                                const int *nl, float *t, cudaStream_t s);
cudaError_t launch_project_init(int conn, const Geom &g, const int *cs, const int *ct, const int *nl, const float *p,
                                int *F, int *ft, cudaStream_t s);
// the trims in one cooperative launch, tile-local phases; flags: 5 ints
// (flags[2] = phases run, 0 if nothing was trimmed, -1: no preflow
// reachable or the phase cap hit)
cudaError_t launch_project_rounds(int conn, const Geom &g, const int *cs, const int *ct, int *F, int *ft, int *E,
                                  int *flags, int max_rounds, cudaStream_t s);
cudaError_t launch_warm_init(int conn, const Geom &g, const DevState &st, const int *cs, const int *ct, const int *nl,
                             const int *F, const int *ft, const int *E, cudaStream_t s);
// brelabel.cu: boundary-relabel heuristic (Sec. 6.1), any grid and tile
struct BrResult {
    int levels;    // levels of the search over the auxiliary graph
    int merged;    // faces whose staircase was shortened (0: d' exact)
    int applied;   // 0: the breakpoint pool overflowed and nothing changed
    int launches;  // kernels launched
};
size_t br_scratch_bytes(const Geom &g, int conn);
// h_words: pinned host buffer of >= 8 ints; leaves st.ctr[kActiveRegions] =
// regions active under the new labels when applied
cudaError_t boundary_relabel(int conn, const Geom &g, const DevState &st, void *scratch, int *h_words,
                             BrResult *res, cudaStream_t s);
// ard_discharge2d.cu
bool discharge2d_supported(int conn, int tx, int ty);
cudaError_t launch_discharge2d_batch(int conn, int tx, int ty, const Inst *insts, const int2 *items,
                                     const int *count, int *head, const SweepArgs &sa, int blocks,
                                     cudaStream_t stream);
cudaError_t launch_discharge2d(int conn, const Geom &g, const DevState &st, const SweepArgs &sa,
                               cudaStream_t stream);
// ard_discharge3d.cu (6-connected, tiles 32x16x8 and 32x8x8)
bool discharge3d_supported(int tx, int ty, int tz);
cudaError_t launch_discharge3d(const Geom &g, const DevState &st, const SweepArgs &sa, cudaStream_t stream);
cudaError_t launch_discharge3d_batch(int tx, int ty, int tz, const Inst *insts, const int2 *items, const int *count,
                                     int *head, const SweepArgs &sa, int blocks, cudaStream_t stream);

}  // namespace mf
