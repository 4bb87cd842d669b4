// psc_internal.h -- plain-data structures passed from the C ABI layer to the kernel
// launchers of the PSC lattice-Boltzmann library. Host-visible; no CUDA device code here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

// Bounds-checked build (compiled with -DPSC_CHECKED; build(checked=True)): the kernels test
// the indices of their main global accesses against the buffer extents. An index out of
// range is recorded as a bit of one device word per translation unit (no relocatable device
// code), read and cleared through lbm_check_violations, and replaced by 0, so the run goes on
// without touching memory outside the buffers (its results are then wrong, and the word
// says so). Unchecked builds compile the tests out: PSC_IDX(i, ...) is i.
enum {
    CHK_POP = 1u,        // population index outside [0, Q N)
    CHK_TILE = 2u,       // tile index outside [0, tiles) or list slot outside its capacity
    CHK_PART = 4u,       // particle index outside [0, n)
    CHK_REC = 8u,        // packed-record word outside the tile's block
    CHK_NBR = 16u,       // DEM neighbour slot or history index outside its list
};
#ifdef PSC_CHECKED
static __device__ unsigned int psc_chk_word;
#define PSC_CHECK(cond, bit) do { if (!(cond)) atomicOr(&psc_chk_word, (unsigned)(bit)); } while (0)
__device__ __forceinline__ long long psc_chk_idx(long long i, long long lim, unsigned bit) {
    if ((unsigned long long)i >= (unsigned long long)lim) { atomicOr(&psc_chk_word, bit); return 0; }
    return i;
}
#define PSC_IDX(i, lim, bit) psc_chk_idx((long long)(i), (long long)(lim), (unsigned)(bit))
// an offset from base index b, checked as the index b + off
#define PSC_OFF(b, off, lim, bit) (PSC_IDX((b) + (off), (lim), (bit)) - (long long)(b))
// the host reader of this translation unit's word (returns it and clears it)
#define PSC_CHECK_READER(name)                                                   \
    unsigned int name() {                                                        \
        unsigned int v = 0, z = 0;                                               \
        if (cudaMemcpyFromSymbol(&v, psc_chk_word, sizeof(v)) != cudaSuccess) return 0xffffffffu; \
        cudaMemcpyToSymbol(psc_chk_word, &z, sizeof(z));                         \
        return v;                                                                \
    }
#else
#define PSC_CHECK(cond, bit) do { } while (0)
#define PSC_IDX(i, lim, bit) (i)
#define PSC_OFF(b, off, lim, bit) (off)
#define PSC_CHECK_READER(name) \
    unsigned int name() { return 0u; }
#endif

namespace psc {

// Lattice geometry and the tiling of the lattice into thread blocks.
struct Geom {
    int n[3];            // nx, ny, nz
    long long ncell;     // nx * ny * nz
    int periodic[3];     // 1 = periodic axis, 0 = another face kind (see faces)
    int wrap_img[3];     // 1 = periodic axis short enough to need a per-cell minimum image
    int nt[3];           // tiles per axis (tile extent: tile_ext)
    int faces;           // what lies beyond each face, a FaceKind in 3 bits per face (face_kind):
                         // a population whose source x - e_i is beyond it wraps, bounces back,
                         // is clamped to the lattice (open face) or is set by the velocity inlet
                         // or the constant-pressure outlet
    double inv_n[3];     // 1 / n per axis (no FP64 division on the device)
    int act0, act1;      // cells updated along the slowest axis (y for D2Q9, z for D3Q19):
                         // act0 <= coordinate < act1 ([0, n) except in a slab of a decomposed
                         // lattice, whose ghost layers are read only)
};
// The kernels take Geom by value next to their other parameters; it is kept this compact
// on purpose (each field added to it measured a few per cent on the collide-stream kernels).
enum FaceKind { FACE_PERIODIC = 0, FACE_WALL = 1, FACE_OPEN = 2, FACE_INFLOW = 3, FACE_OUTLET = 4 };
// Kind of the low (hi = 0) or high (hi = 1) face of axis a.
__host__ __device__ inline int face_kind(const Geom &g, const int a, const int hi) {
    return (g.faces >> (6 * a + 3 * hi)) & 7;
}
__host__ inline void set_face_kind(Geom &g, const int a, const int hi, const int kind) {
    const int sh = 6 * a + 3 * hi;
    g.faces = (g.faces & ~(7 << sh)) | (kind << sh);
}
// Tile extent along axis ax: 32 x 8 x 1 cells for D2Q9, 32 x 4 x 2 for D3Q19 (one tile is
// one thread block of the single-cell kernels).
__host__ __device__ inline int tile_ext(const int dim, const int ax) {
    return dim == 2 ? (ax == 0 ? 32 : (ax == 1 ? 8 : 1)) : (ax == 0 ? 32 : (ax == 1 ? 4 : 2));
}

// Physical parameters (FP64 on the host; kernels convert to their compute type).
struct Phys {
    double tau;
    double body_force[3];
    double shell_h;      // h of Table 1
    double scale;        // stored value = scale * (f_i - w_i); 1 except for FP16/BF16
    int psc;             // 0 modified (Eq. 12-14), 1 original (Eq. 7-9, 11)
    double inflow[3];    // velocity imposed on the inlet face
    int inflow_axis;     // axis whose low face is the inlet, -1 when there is none
};

// Per-tile candidate lists built by the binning kernel: count[tile] particles whose
// (r + h)-widened bounding box meets the tile; the first `cap` of them in list[tile*cap+k].
struct Tiles {
    int *count;
    int *list;
    int cap;
    int *stats;          // [0] tiles that overflowed cap, [1] largest count, [2] length of
                         // the overflow list, [3] [6] work counters of the collide-stream
                         // kernel over the fluid and the particle tiles (zero between
                         // launches), [4] tiles with candidates, [5] tiles without
    void *blocks;        // per-tile packed candidate records (compute type), see psc_kernels.cuh
    uint2 *order;        // [3 * ntiles] {tile id, ty | tz << 16}: tiles with candidates, then
                         // (from ntiles on) tiles without, then (from 2 ntiles on) tiles with
                         // more than cap; each list in rising id order within a block of 8
};
constexpr int kTileStats = 8;

// Particle state on the device (FP64), and the force/torque accumulators (Eq. 14).
struct Parts {
    int n;
    const double *X, *U, *Om, *R, *Fr;   // n x 3, n x 3, n x 3, n, n (f(r) of Eq. 18)
    double *F, *T;                       // n x 3 each
    float4 *Pf;                          // optional [n][2]: {r, f(r), Ux, Uy}, {Uz, Ox, Oy, Oz} in
                                         // FP32, written by the binning kernel for the records
};

enum StorageKind { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };

// A second stream and two events, for the two kernels of a step that run side by side
// (forked from the caller's stream and joined back into it). Null: one stream.
struct Overlap {
    cudaStream_t aux;
    cudaEvent_t fork, join;
    // defer = 1 (a coupled step, whose DEM call follows on the main stream): where the
    // particle and plain-fluid tiles run on two streams, the particle tiles (and the overflow
    // tiles) run first at full occupancy, the fluid tiles follow on aux with room left on
    // every SM for the main stream's next kernels, and the join is left to the caller, who
    // waits on `join` when the launcher sets deferred = 1
    int defer, deferred;
    // recorded on aux by a coupled step once the DEM call's preparation kernels (which read
    // only the particle state the fluid step leaves alone) have run there
    cudaEvent_t prep;
};

// Fused solid-fraction + PSC collision + pull streaming + force reduction (one step).
cudaError_t launch_collide_stream(int storage, int lattice, const void *fin, void *fout,
                                  const Geom &g, const Phys &ph, const Tiles &tl,
                                  const Parts &pd, int *flags, cudaStream_t s, Overlap *ov);
// Pre-collision populations (full f, FP64) and/or Eq. 5 moments of the current state.
cudaError_t launch_gather(int storage, int lattice, const void *fin, double *f_out,
                          double *rho, double *u, const Geom &g, const Phys &ph,
                          cudaStream_t s);
// Overwrite the state from pre-collision populations (inverse of the pull).
cudaError_t launch_set(int storage, int lattice, const double *f, void *fout,
                       const Geom &g, const Phys &ph, cudaStream_t s);
// Bin particles into tile candidate lists and zero F, T.
cudaError_t launch_bin(int dim, const Geom &g, const Phys &ph, const Tiles &tl,
                       const Parts &pd, cudaStream_t s);
// Sort each tile's list and write its packed candidate records (rec_double: FP64 records).
cudaError_t launch_pack(int lattice, int rec_double, const Geom &g, const Tiles &tl, const Parts &pd,
                        long long ntiles, cudaStream_t s);
// Bytes of one tile's packed block for the given candidate capacity.
long long pack_block_bytes(int rec_double, int cap);
// One reverse step of the collide-stream step (static particles): lam_out = S^T (dC/dp)^T
// lam_in + drag terms; accumulates dJ/dX (n x 3, atomics) and per-block partials of dJ/dF
// (blocks x 3, each block adds to its own slot).
cudaError_t launch_adjoint(int storage, int lattice, const void *gt, const void *lam_in, void *lam_out,
                           const Geom &g, const Phys &ph, const Tiles &tl, const Parts &pd, double invT,
                           double *dJdX, double *dFpart, cudaStream_t s);
// f(r) of Eq. 18 (Eq. 17 in 3D, Eq. 19 in 2D) for every particle.
cudaError_t launch_f_of_r(int dim, const double *R, double *Fr, int n, cudaStream_t s);
// A particle upload in one launch: X, U, Omega (n x 3) and the radii copied from the
// sources (device memory, or page-locked host memory mapped into the device's address
// space; a source may be its own destination) into the context's arrays, F and T cleared,
// f(r) evaluated; when `ref` is set, *req = 1 if some particle lies more than sqrt(lim2)
// (FP32, one image shift on periodic axes) from its reference position.
struct Upload {
    const double *X, *U, *Om, *R;
    double *dX, *dU, *dOm, *dR, *dFr, *dF, *dT;
    int n, dim;
    const double *ref;
    int *req;
    float lim2;
    int n_lat[3], periodic[3];
};
cudaError_t launch_upload(const Upload &u, cudaStream_t s);
// m = 3 n doubles of F and T (either output may be NULL) and the four flag words copied to
// the caller's memory (device memory or mapped page-locked host memory).
cudaError_t launch_download(const double *F, const double *T, double *Fo, double *To, long long m,
                            const int *flags, int *flags_out, cudaStream_t s);

}  // namespace psc
