// psc_kernels.cuh -- sm_103a kernels of one lattice-Boltzmann step with the modified
// partially-saturated-cell (PSC) immersed moving boundary (Liu & Wu, arXiv 1901.09745).
//
// The lattice is cut into tiles (32 x 8 cells in 2D, 32 x 4 x 2 in 3D). After binning,
// k_pack_tiles writes each tile's candidate particles as packed records and sorts the
// tiles into three lists: tiles without candidates (k_fluid_pair: BGK + Guo + pull only),
// tiles with at most 32 (k_collide_stream, psc_pair.cuh), tiles with more (the exact
// chunked path of k_collide_overflow, psc_tile below). Per cell every path
//   1. pulls the Q post-collision populations of the previous step from the neighbours
//      x - e_i (Eq. 1; periodic wrap; halfway bounce-back at walls, Eq. 6),
//   2. forms rho and the force-shifted u (Eq. 5),
//   3. walks the tile's candidate particles held in shared memory and computes each
//      particle's solid fraction by the linear approximation (Eq. 15-18, Table 1),
//   4. forms eps_n, B_n (Eq. 9) and the per-particle weights B_{n,s} (Eq. 13),
//   5. collides with BGK + Guo forcing + sum_s B_{n,s} Omega^s (Eq. 2-4, 10, 12) and
//      stores the Q post-collision populations of its own cell,
//   6. reduces each particle's momentum exchange B_{n,s} sum_i Omega^s_i e_i and its
//      torque (Eq. 14) over the warp with shuffles, over the block in shared memory, and
//      adds the block's total with one FP64 atomic per particle and component.
//
// Two algebraic identities keep the per-candidate work independent of Q (exact up to
// rounding order, derived from Eq. 3 and Eq. 10):
//   sum_s B_{n,s} f_i^eq(rho, u_s) = rho w_i [B_n + 3 e_i.m + 9/2 e_i.M.e_i - 3/2 tr M],
//       m = sum_s B_{n,s} u_s, M = sum_s B_{n,s} u_s u_s^T   (f^eq is quadratic in u_s);
//   sum_i Omega^s_i e_i = rho (u + u_s) - 2 j = rho u_s + F/2 - j,   j = sum_i f_i e_i.
// Populations are stored as deviations d_i = f_i - w_i, so every stored and summed value
// is small and FP32 keeps its relative precision (rho = 1 + sum_i d_i).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
#include "hostdev.cuh"
#include "psc_internal.h"

namespace psc {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kPairCap = 32;     // candidates a tile may have to take the two-cells-per-thread path

template <typename T> struct PhysT {
    T omega;        // 1/tau
    T tmh;          // tau - 1/2
    T guo;          // 1 - 1/(2 tau), Eq. 4
    T F[3];         // body force
    T h;            // Table 1 shell half-width
    float2 sc;      // (scale, 1/scale) of the stored deviations
    int inax;       // axis whose low face is an inlet (-1: none)
    T inua;         // inlet velocity along that axis
    T ineu[19];     // 6 w_i (e_i . u_in): f^eq_i - f^eq_{-i} of Eq. 3 at rho = 1
};

template <typename T> __host__ PhysT<T> make_phys(const Phys &ph, const int lattice = 19) {
    PhysT<T> k;
    k.omega = (T)(1.0 / ph.tau);
    k.tmh = (T)(ph.tau - 0.5);
    k.guo = (T)(1.0 - 1.0 / (2.0 * ph.tau));
    for (int a = 0; a < 3; ++a) k.F[a] = (T)ph.body_force[a];
    k.h = (T)ph.shell_h;
    k.sc = make_float2((float)ph.scale, (float)(1.0 / ph.scale));
    const double *u = ph.inflow;
    k.inax = ph.inflow_axis;
    k.inua = (T)(ph.inflow_axis >= 0 ? u[ph.inflow_axis] : 0.0);   // the inlet is a low face
    for (int i = 0; i < 19; ++i) {
        double eu = 0.0, w = 0.0;
        if (lattice == 9 && i < 9) { eu = D2Q9::ex(i) * u[0] + D2Q9::ey(i) * u[1]; w = weight<D2Q9>(i); }
        else if (lattice == 19) { eu = D3Q19::ex(i) * u[0] + D3Q19::ey(i) * u[1] + D3Q19::ez(i) * u[2]; w = weight<D3Q19>(i); }
        k.ineu[i] = (T)(6.0 * w * eu);
    }
    return k;
}

// Velocity inlet (reading of Sec. 3.2's "constant flow with velocity U0"): on the inlet face
// the populations coming in (e_a = +1 along the inlet axis a) are not known from a
// neighbour; they take the non-equilibrium part of the opposite population, f_i = f_{-i} +
// f^eq_i(rho, u_in) - f^eq_{-i}(rho, u_in) = f_{-i} + 6 w_i rho e_i.u_in, with the density that
// gives the face cell the velocity u_in along a: rho (1 - u_a) = sum_{e_a = 0} f + 2 sum_{e_a = -1} f.
// df holds deviations (scaled by s when RAW); the directions in `fill` (those whose source
// lies beyond the inlet and beyond no wall) are overwritten.
template <class L, bool RAW, typename T>
__device__ __forceinline__ void inflow_nebb(T *df, const PhysT<T> &ph, const float2 sc, const unsigned fill) {
    const int a = ph.inax;
    T sd = (T)0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int ea = (a == 0) ? L::ex(i) : ((a == 1) ? L::ey(i) : L::ez(i));
        if (ea == 0) sd += df[i];
        else if (ea == -1) sd += (T)2 * df[i];
    }
    const T s = RAW ? (T)sc.x : (T)1;
    // sum_{e_a = 0} w + 2 sum_{e_a = -1} w = 1, so the deviations give rho directly
    const T rho = ((T)1 + sd / s) / ((T)1 - ph.inua);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        if (fill & (1u << i)) df[i] = df[opp<L>(i)] + s * rho * ph.ineu[i];
    }
}

// Constant-pressure outlet (reading of Sec. 3.2's outlet), on the high face of the inlet axis
// a: the populations coming in (e_a = -1) are unknown; the density is held at 1 and the
// velocity across the face follows from the known ones, 1 + u_a = sum_{e_a = 0} f +
// 2 sum_{e_a = +1} f; the unknown ones are f_i = f_{-i} + 6 w_i e_{i,a} u_a (the difference of
// the equilibria of Eq. 3 at rho = 1, u = u_a along a).
template <class L, bool RAW, typename T>
__device__ __forceinline__ void outlet_nebb(T *df, const PhysT<T> &ph, const float2 sc, const unsigned fill) {
    const int a = ph.inax;
    T sd = (T)0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int ea = (a == 0) ? L::ex(i) : ((a == 1) ? L::ey(i) : L::ez(i));
        if (ea == 0) sd += df[i];
        else if (ea == 1) sd += (T)2 * df[i];
    }
    // sum_{e_a = 0} w + 2 sum_{e_a = +1} w = 1: the scaled deviation sum is s u_a
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int ea = (a == 0) ? L::ex(i) : ((a == 1) ? L::ey(i) : L::ez(i));
        if (fill & (1u << i)) df[i] = df[opp<L>(i)] + (T)(6.0 * weight<L>(i)) * (T)ea * sd;
    }
    (void)sc;
}

// Programmatic dependent launch within the step: a kernel launched with launch_pdl may start
// while its predecessor in the stream finishes; it calls pdl_wait() before it reads anything
// the predecessor wrote, and pdl_launch() lets its own successor start early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Is cell (x, y, z) one this context updates (inside the lattice and, in a slab of a
// decomposed lattice, outside its ghost layers along the slowest axis; act1 <= n there)?
template <class L>
__device__ __forceinline__ bool cell_active(const Geom &g, const int x, const int y, const int z) {
    if (L::D == 2) return x < g.n[0] && (unsigned)(y - g.act0) < (unsigned)(g.act1 - g.act0);
    return x < g.n[0] && y < g.n[1] && (unsigned)(z - g.act0) < (unsigned)(g.act1 - g.act0);
}

__device__ __forceinline__ float  rint_t(float v) { return rintf(v); }
__device__ __forceinline__ double rint_t(double v) { return rint(v); }
__device__ __forceinline__ float  sqrt_t(float v) { return sqrtf(v); }
__device__ __forceinline__ double sqrt_t(double v) { return sqrt(v); }
// Distances of cells from particle centres in the solid-fraction and row tests: FP32 takes
// v * rsqrt(v) (a few ulp, far below the FP32 parity tolerance; two instructions instead of
// the correctly rounded square root); FP64 keeps the correctly rounded one.
__device__ __forceinline__ float  dist_t(float v) { return v > 0.0f ? v * rsqrtf(v) : 0.0f; }
__device__ __forceinline__ double dist_t(double v) { return sqrt(v); }

// Population i of cell (x, y, z) after streaming: the value the neighbour x - e_i stored
// in the previous step, or, when x - e_i lies beyond a wall, the value this cell stored in
// the opposite direction (halfway bounce-back, Eq. 6). Periodic and wall faces only.
template <class L, typename S>
__device__ __forceinline__ typename Store<S>::T
pull_one(const S *__restrict__ fin, const Geom &g, int x, int y, int z, long long cell, int i,
         float2 sc) {
    int s[3] = {x - L::ex(i), y - L::ey(i), z - L::ez(i)};
    bool bounce = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (s[a] < 0 || s[a] >= g.n[a]) {
            if (g.periodic[a]) s[a] += (s[a] < 0) ? g.n[a] : -g.n[a];
            else bounce = true;
        }
    }
    if (bounce) return Store<S>::ld(fin, PSC_IDX((long long)opp<L>(i) * g.ncell + cell, L::Q * g.ncell, CHK_POP), sc);
    long long src = (long long)s[0] + (long long)g.n[0] * ((long long)s[1] + (long long)g.n[1] * s[2]);
    return Store<S>::ld(fin, PSC_IDX((long long)i * g.ncell + src, L::Q * g.ncell, CHK_POP), sc);
}

// The same for every face kind: beyond an open face the source is clamped onto the face
// (zero gradient); beyond the inlet or the outlet face the population is unknown (returned
// as 0, `from_inlet` or `from_outlet` set) and is filled in by inflow_nebb or outlet_nebb
// once all are pulled. A wall takes precedence over the inlet and outlet faces, these over
// open faces.
template <class L, typename S>
__device__ __forceinline__ typename Store<S>::T
pull_one_faces(const S *__restrict__ fin, const Geom &g, int x, int y, int z, long long cell, int i,
               float2 sc, bool &from_inlet, bool &from_outlet) {
    int s[3] = {x - L::ex(i), y - L::ey(i), z - L::ez(i)};
    bool bounce = false, inflow = false, outflow = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (s[a] < 0 || s[a] >= g.n[a]) {
            const int kind = face_kind(g, a, s[a] < 0 ? 0 : 1);
            if (kind == FACE_PERIODIC) s[a] += (s[a] < 0) ? g.n[a] : -g.n[a];
            else if (kind == FACE_WALL) bounce = true;
            else if (kind == FACE_OPEN) s[a] = (s[a] < 0) ? 0 : g.n[a] - 1;
            else if (kind == FACE_INFLOW) inflow = true;
            else outflow = true;
        }
    }
    if (bounce) return Store<S>::ld(fin, PSC_IDX((long long)opp<L>(i) * g.ncell + cell, L::Q * g.ncell, CHK_POP), sc);
    from_inlet = inflow;
    from_outlet = outflow && !inflow;
    if (inflow || outflow) return (typename Store<S>::T)0;
    long long src = (long long)s[0] + (long long)g.n[0] * ((long long)s[1] + (long long)g.n[1] * s[2]);
    return Store<S>::ld(fin, PSC_IDX((long long)i * g.ncell + src, L::Q * g.ncell, CHK_POP), sc);
}

// All Q populations of cell (x, y, z) after streaming, one pull_one per direction, the
// unknown ones at an inlet filled in.
template <class L, typename S>
__device__ __forceinline__ void pull_all(const S *__restrict__ fin, const Geom &g, int x, int y, int z,
                                         long long cell, const PhysT<typename Store<S>::T> &ph,
                                         typename Store<S>::T *df) {
    unsigned fill = 0u, fillo = 0u;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        bool in = false, out = false;
        df[i] = pull_one_faces<L, S>(fin, g, x, y, z, cell, i, ph.sc, in, out);
        if (in) fill |= 1u << i;
        if (out) fillo |= 1u << i;
    }
    if (fill) inflow_nebb<L, false>(df, ph, ph.sc, fill);
    if (fillo) outlet_nebb<L, false>(df, ph, ph.sc, fillo);
}

// Warp sum of NV values per lane (NV a power of two <= 32) in NV - 1 + 5 - log2(NV) shuffles
// instead of 5 NV: each butterfly stage first halves the set of values a lane carries (it
// keeps one half and sends the other to its partner), then plain butterflies finish. On
// return lane l holds the warp total of value l >> (5 - log2 NV).
template <int NV, typename T>
__device__ __forceinline__ T warp_sum_spread(T (&v)[NV], const int lane) {
    int m = NV;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        if (m > 1) {
            const int half = m >> 1;
            const bool up = (lane & off) != 0;
#pragma unroll
            for (int j = 0; j < NV / 2; ++j) {
                if (j < half) {
                    const T snd = up ? v[j] : v[j + half];
                    const T kp = up ? v[j + half] : v[j];
                    v[j] = kp + __shfl_xor_sync(kFull, snd, off);
                }
            }
            m = half;
        } else {
            v[0] += __shfl_xor_sync(kFull, v[0], off);
        }
    }
    return v[0];
}

// e_i . v for a lattice velocity with components in {-1, 0, 1}: additions only, no
// multiplications by 0 or 1 (which IEEE arithmetic does not let the compiler drop).
template <class L, typename T>
__device__ __forceinline__ T edot(const int i, const T vx, const T vy, const T vz) {
    const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
    T r = (T)0;
    bool first = true;
    if (ex) { r = ex > 0 ? vx : -vx; first = false; }
    if (ey) { r = first ? (ey > 0 ? vy : -vy) : (ey > 0 ? r + vy : r - vy); first = false; }
    if (ez) { r = first ? (ez > 0 ? vz : -vz) : (ez > 0 ? r + vz : r - vz); }
    return r;
}

// Where the pull of direction i at cell x reads (Eq. 1, 6): x - e_i, or the cell itself in
// direction -i when x - e_i lies beyond a wall (halfway bounce-back). The offsets to the -1
// and +1 neighbour on each axis (periodic wrap folded in) and the wall flags are formed once
// per cell, so each direction costs an add and a select instead of three range tests. The
// adjoint pushes to the same index.
struct NbrIdx {
    long long oxm, oxp, oym, oyp, ozm, ozp;   // source offsets when e = +1 (m) / -1 (p)
    unsigned wall;                            // bits 0..5: wxm wxp wym wyp wzm wzp
};

template <class L>
__device__ __forceinline__ NbrIdx make_nbr_idx(const Geom &g, int x, int y, int z) {
    const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
    NbrIdx nb{-1, 1, -sy, sy, -sz, sz, 0u};
    if (x == 0) { if (g.periodic[0]) nb.oxm = g.n[0] - 1; else nb.wall |= 1u; }
    if (x == g.n[0] - 1) { if (g.periodic[0]) nb.oxp = -(long long)(g.n[0] - 1); else nb.wall |= 2u; }
    if (y == 0) { if (g.periodic[1]) nb.oym = (long long)(g.n[1] - 1) * sy; else nb.wall |= 4u; }
    if (y == g.n[1] - 1) { if (g.periodic[1]) nb.oyp = -(long long)(g.n[1] - 1) * sy; else nb.wall |= 8u; }
    if (L::D == 3) {
        if (z == 0) { if (g.periodic[2]) nb.ozm = (long long)(g.n[2] - 1) * sz; else nb.wall |= 16u; }
        if (z == g.n[2] - 1) { if (g.periodic[2]) nb.ozp = -(long long)(g.n[2] - 1) * sz; else nb.wall |= 32u; }
    }
    return nb;
}

template <class L>
__device__ __forceinline__ long long src_index(const NbrIdx &nb, const int i, const long long cell, const long long N) {
    long long off = 0;
    unsigned w = 0u;
    if (L::ex(i) == 1) { off += nb.oxm; w |= 1u; }
    if (L::ex(i) == -1) { off += nb.oxp; w |= 2u; }
    if (L::ey(i) == 1) { off += nb.oym; w |= 4u; }
    if (L::ey(i) == -1) { off += nb.oyp; w |= 8u; }
    if (L::ez(i) == 1) { off += nb.ozm; w |= 16u; }
    if (L::ez(i) == -1) { off += nb.ozp; w |= 32u; }
    return (nb.wall & w) ? (long long)opp<L>(i) * N + cell : (long long)i * N + cell + off;
}

// All Q pulled deviations of the cell (x, y, z). Tiles one cell clear of every face use
// fixed offsets; elsewhere the same offsets and wall flags as make_nbr_idx, held in scalars
// (measured faster here than going through the struct).
template <class L, typename S, bool RAW = false>
__device__ __forceinline__ void pull_q(const S *__restrict__ fin, const Geom &g, int x, int y, int z,
                                       long long cell, bool interior, bool active, float2 sc,
                                       typename Store<S>::T *df) {
    constexpr int Q = L::Q;
    using T = typename Store<S>::T;
    const long long N = g.ncell;
    const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
    if (interior) {
        const S *base = fin + cell;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const long long o = (long long)i * N - (L::ex(i) + L::ey(i) * sy + L::ez(i) * sz);
            const long long oc = PSC_OFF(cell, o, Q * N, CHK_POP);
            df[i] = RAW ? Store<S>::ldr(base, oc) : Store<S>::ld(base, oc, sc);
        }
        return;
    }
    if (!active) {
#pragma unroll
        for (int i = 0; i < Q; ++i) df[i] = (T)0;
        return;
    }
    // source x - e: from the -1 neighbour when e = +1 (m), from the +1 neighbour when e = -1 (p);
    // periodic and wall faces only (contexts with open, inlet or outlet faces step with
    // k_collide_faces)
    long long oxm = -1, oxp = 1, oym = -sy, oyp = sy, ozm = -sz, ozp = sz;
    bool wxm = false, wxp = false, wym = false, wyp = false, wzm = false, wzp = false;
    if (x == 0) { if (g.periodic[0]) oxm = g.n[0] - 1; else wxm = true; }
    if (x == g.n[0] - 1) { if (g.periodic[0]) oxp = -(long long)(g.n[0] - 1); else wxp = true; }
    if (y == 0) { if (g.periodic[1]) oym = (long long)(g.n[1] - 1) * sy; else wym = true; }
    if (y == g.n[1] - 1) { if (g.periodic[1]) oyp = -(long long)(g.n[1] - 1) * sy; else wyp = true; }
    if (L::D == 3) {
        if (z == 0) { if (g.periodic[2]) ozm = (long long)(g.n[2] - 1) * sz; else wzm = true; }
        if (z == g.n[2] - 1) { if (g.periodic[2]) ozp = -(long long)(g.n[2] - 1) * sz; else wzp = true; }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        long long off = 0;
        bool wall = false;
        if (L::ex(i) == 1) { off += oxm; wall |= wxm; }
        if (L::ex(i) == -1) { off += oxp; wall |= wxp; }
        if (L::ey(i) == 1) { off += oym; wall |= wym; }
        if (L::ey(i) == -1) { off += oyp; wall |= wyp; }
        if (L::ez(i) == 1) { off += ozm; wall |= wzm; }
        if (L::ez(i) == -1) { off += ozp; wall |= wzp; }
        const long long idx = wall ? (long long)opp<L>(i) * N + cell : (long long)i * N + cell + off;
        const long long ic = PSC_IDX(idx, Q * N, CHK_POP);
        df[i] = RAW ? Store<S>::ldr(fin, ic) : Store<S>::ld(fin, ic, sc);
    }
}

// ------------------------------------------------------------------- candidate records
// Each lattice tile owns one block of candidate records in global memory, written by the
// packing kernel after binning: a 16-byte header whose first element is the tile's
// candidate count, then up to `cap` records of RW values of the compute type, sorted by
// particle index (so per-cell sums do not depend on the binning's atomic order). A record
// holds the particle's position relative to the tile origin (minimum image), radius,
// f(r) of Eq. 18, velocity, spin and index. The collide-stream kernel fetches a tile's
// header and first kPre records in one coalesced round trip issued before its population
// loads, so the candidate table costs no extra latency on the critical path.
constexpr int RW = 12;
enum { R_PX = 0, R_PY, R_PZ, R_R, R_FR, R_UX, R_UY, R_UZ, R_OX, R_OY, R_OZ, R_ID };
constexpr int kPre = 16;

template <typename T> __host__ __device__ constexpr int head_elems() { return 16 / (int)sizeof(T); }
template <typename T> __host__ __device__ inline long long block_elems(int cap) {
    return ((head_elems<T>() + (long long)cap * RW + 3) / 4) * 4;
}
template <typename T> __host__ __device__ inline size_t cs_smem_bytes(int cap, int nc) {
    return (size_t)cap * RW * sizeof(T) + (size_t)kWarps * cap * nc * sizeof(T);
}

// Particle index stored in a record slot as raw bits (no conversion instruction).
template <typename T> __device__ __forceinline__ T id_bits(int id);
template <> __device__ __forceinline__ float id_bits<float>(int id) { return __int_as_float(id); }
template <> __device__ __forceinline__ double id_bits<double>(int id) { return __longlong_as_double((long long)id); }
__device__ __forceinline__ int bits_id(float v) { return __float_as_int(v); }
__device__ __forceinline__ int bits_id(double v) { return (int)__double_as_longlong(v); }

// Record of particle `id` for the tile with origin (x0, y0, z0).
template <class L, typename T>
__device__ __forceinline__ void write_record(T *rec, const Geom &g, const Parts &pd, int id, int x0,
                                             int y0, int z0) {
    const int org[3] = {x0, y0, z0};
    const int ext[3] = {L::TX, L::TY, L::TZ};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T rel = (T)0;
        if (a < L::D) {
            // minimum image with respect to the tile centre, one exact FP64 subtraction
            rel = (T)record_rel(pd.X[3 * id + a], org[a], ext[a], g.n[a], g.inv_n[a], g.periodic[a]);
        }
        rec[R_PX + a] = rel;
    }
    if (sizeof(T) == 4 && pd.Pf) {   // FP32 records: the per-particle copy, no conversions here
        const float4 a = pd.Pf[2 * id], b = pd.Pf[2 * id + 1];
        rec[R_R] = (T)a.x; rec[R_FR] = (T)a.y;
        rec[R_UX] = (T)a.z; rec[R_UY] = (T)a.w; rec[R_UZ] = (T)b.x;
        rec[R_OX] = (T)b.y; rec[R_OY] = (T)b.z; rec[R_OZ] = (T)b.w;
    } else {
        rec[R_R] = (T)pd.R[id];
        rec[R_FR] = (T)pd.Fr[id];
        rec[R_UX] = (T)pd.U[3 * id + 0]; rec[R_UY] = (T)pd.U[3 * id + 1]; rec[R_UZ] = (T)pd.U[3 * id + 2];
        rec[R_OX] = (T)pd.Om[3 * id + 0]; rec[R_OY] = (T)pd.Om[3 * id + 1]; rec[R_OZ] = (T)pd.Om[3 * id + 2];
    }
    rec[R_ID] = id_bits<T>(id);
}

// Packing kernel: one warp per tile sorts the tile's candidate list and writes its block.
// Each block of 8 tiles then appends its tiles to the list of tiles with candidates or to
// the list of tiles without, and tiles with more candidates than `cap` also to the overflow
// list (tiles with more than min(cap, kPairCap) candidates; one atomic per list and block), so
// the collide-stream kernels run over compact lists and launch no block for a tile that is
// not theirs.
template <class L, typename T>
__global__ void k_pack_tiles(Geom g, Tiles tl, Parts pd, long long ntiles) {
    __shared__ int s_id[kWarps][64];
    __shared__ int s_cnt[kWarps];
    __shared__ uint2 s_ent[kWarps];
    pdl_wait();       // the binning kernel's counts and lists
    pdl_launch();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // grid (nt0 / 8, nt1, nt2): the block's 8 warps take 8 tiles along x, no division
    const int tx = (int)blockIdx.x * kWarps + warp, ty = (int)blockIdx.y, tz = (int)blockIdx.z;
    const long long tile = tx + (long long)g.nt[0] * (ty + (long long)g.nt[1] * tz);
    const bool valid = tx < g.nt[0];
    const int cnt = valid ? tl.count[tile] : -1;
    if (lane == 0) s_cnt[warp] = cnt;
    if (valid) {
        const int m = min(cnt, tl.cap);
        T *blk = reinterpret_cast<T *>(tl.blocks) + tile * block_elems<T>(tl.cap);
        if (lane == 0) blk[0] = (T)cnt;
        for (int k = lane; k < m; k += 32) s_id[warp][k] = tl.list[tile * tl.cap + k];
        __syncwarp();
        if (lane == 0) s_ent[warp] = make_uint2((unsigned)tile, (unsigned)ty | ((unsigned)tz << 16));
        for (int k = lane; k < m; k += 32) {
            const int id = (int)PSC_IDX(s_id[warp][k], pd.n, CHK_PART);
            int rank = 0;
            for (int q = 0; q < m; ++q) rank += (s_id[warp][q] < id);
            write_record<L, T>(blk + head_elems<T>() + (long long)rank * RW, g, pd, id, tx * L::TX, ty * L::TY,
                               tz * L::TZ);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int np = 0, nf = 0;
        for (int w = 0; w < kWarps; ++w) { np += (s_cnt[w] > 0); nf += (s_cnt[w] == 0); }
        int no = 0;
        const int lim = min(tl.cap, kPairCap);
        for (int w = 0; w < kWarps; ++w) no += (s_cnt[w] > lim);
        int bp = np ? atomicAdd(&tl.stats[4], np) : 0;
        int bf = nf ? atomicAdd(&tl.stats[5], nf) : 0;
        int bo = no ? atomicAdd(&tl.stats[2], no) : 0;
        for (int w = 0; w < kWarps; ++w) {
            if (s_cnt[w] < 0) continue;
            const uint2 ent = s_ent[w];
            if (s_cnt[w] > 0) tl.order[bp++] = ent;
            else tl.order[ntiles + bf++] = ent;
            if (s_cnt[w] > lim) tl.order[2 * ntiles + bo++] = ent;
        }
    }
}

// The geometric part of a record (position, radius) and the rest (f(r), U, Omega, index),
// read from shared memory with 16-byte loads (records are 16-byte aligned).
template <typename T> struct Vec4 { T x, y, z, w; };
template <typename T> __device__ __forceinline__ Vec4<T> ld4(const T *p);
template <> __device__ __forceinline__ Vec4<float> ld4<float>(const float *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
template <> __device__ __forceinline__ Vec4<double> ld4<double>(const double *p) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    return {a.x, a.y, b.x, b.y};
}

// Solid fraction of the candidate in record `rec` at the cell with tile-relative centre
// (cx, cy, cz): Table 1 Steps 2-4 with the inside/outside branches as stated in Sec. 2.4
// (distance <= r - h -> 1, >= r + h -> 0), else clamp(f(r) - D, 0, 1) with D = distance - r
// (Eq. 15). Returns 0 outside; on return (dx, dy, dz) is the arm x_n - X_p.
template <class L, typename T>
__device__ __forceinline__ T cand_eps(const T *rec, const Geom &g, T cx, T cy, T cz, T h, T &dx, T &dy,
                                      T &dz) {
    const Vec4<T> pr = ld4<T>(rec);                      // px, py, pz, r
    dx = cx - pr.x;
    dy = cy - pr.y;
    dz = (L::D == 3) ? cz - pr.z : (T)0;
    if (g.wrap_img[0]) dx -= (T)g.n[0] * rint_t(dx / (T)g.n[0]);
    if (g.wrap_img[1]) dy -= (T)g.n[1] * rint_t(dy / (T)g.n[1]);
    if (L::D == 3 && g.wrap_img[2]) dz -= (T)g.n[2] * rint_t(dz / (T)g.n[2]);
    const T d2 = dx * dx + dy * dy + dz * dz;
    const T r = pr.w;
    const T rh = r + h;
    if (!(d2 < rh * rh)) return (T)0;
    const T dist = sqrt_t(d2);
    if (dist <= r - h) return (T)1;
    T e = rec[R_FR] - (dist - r);
    e = e < (T)0 ? (T)0 : e;
    e = e > (T)1 ? (T)1 : e;
    return e;
}

// Arm x_n - X_p from the cell (cx, cy, cz) to the candidate at (px, py, pz), all relative
// to the tile origin, with the per-cell minimum image on short periodic axes.
template <class L, typename T>
__device__ __forceinline__ void cand_arm(const Geom &g, T cx, T cy, T cz, T px, T py, T pz, T &dx, T &dy,
                                         T &dz) {
    dx = cx - px;
    dy = cy - py;
    dz = (L::D == 3) ? cz - pz : (T)0;
    if (g.wrap_img[0]) dx -= (T)g.n[0] * rint_t(dx / (T)g.n[0]);
    if (g.wrap_img[1]) dy -= (T)g.n[1] * rint_t(dy / (T)g.n[1]);
    if (L::D == 3 && g.wrap_img[2]) dz -= (T)g.n[2] * rint_t(dz / (T)g.n[2]);
}

// Table 1 Steps 2-4 for a cell at squared distance d2 from a candidate of radius r:
// distance <= r - h -> 1, >= r + h -> 0, else clamp(f(r) - D, 0, 1) with D = distance - r.
template <typename T>
__device__ __forceinline__ T shell_eps(T d2, T r, T fr, T h) {
    const T rh = r + h;
    if (!(d2 < rh * rh)) return (T)0;
    const T ri = r - h;
    if (ri > (T)0 && d2 <= ri * ri) return (T)1;
    const T dist = dist_t(d2);
    if (dist <= ri) return (T)1;
    T e = fr - (dist - r);
    e = e < (T)0 ? (T)0 : e;
    e = e > (T)1 ? (T)1 : e;
    return e;
}

// Can the candidate at (px, py, pz) with reach R = r + h touch any cell of this warp's row
// (tile-relative y = cy, z = cz, x = 0..xmax)? Conservative: a false "yes" only costs time.
template <class L, typename T>
__device__ __forceinline__ bool row_hits(const Geom &g, T px, T py, T pz, T R, T cy, T cz, T xmax) {
    T dx, dy, dz;
    cand_arm<L, T>(g, (T)0, cy, cz, (T)0, py, pz, dx, dy, dz);
    const T rem = R * R - dy * dy - dz * dz;
    if (!(rem > (T)0)) return false;
    if (g.wrap_img[0]) return true;
    const T hw = dist_t(rem);
    return (px - hw <= xmax + (T)1) && (px + hw >= (T)-1);
}

template <class L, typename T> constexpr int psc_min_blocks() {
    return sizeof(T) == 8 ? 1 : (L::Q == 9 ? 4 : 3);
}

// Tiles with candidate particles. The tile's records are staged in shared memory while the
// population loads are in flight. Each warp is one row of the tile: it culls the candidates
// that cannot reach its row (one lane per candidate, ballot), then every lane evaluates the
// remaining ones from shared memory (broadcast reads). Warps with no solid cell run the plain
// BGK + Guo update. Forces: each warp reduces each of its candidates' momentum exchange with
// shuffles; partial sums meet in shared memory and are added in a fixed order, one FP64
// atomic per particle and component per tile. Tiles with more candidates than the block
// holds take the same path chunk by chunk over all particles (exact, slow, rare).
template <class L, typename S, int PSC, bool FACES = false>
__device__ __forceinline__ void psc_tile(const unsigned tile, const S *__restrict__ fin, S *__restrict__ fout,
                                         const Geom &g, const PhysT<typename Store<S>::T> &ph, const Tiles &tl,
                                         const Parts &pd, int *flags, typename Store<S>::T *srec,
                                         unsigned long long *s_mask) {
    using T = typename Store<S>::T;
    constexpr int Q = L::Q;
    constexpr int NC = (L::D == 2) ? 3 : 6;
    constexpr int NSLOT = 4;
    const int cap = tl.cap;
    T *part = srec + (size_t)cap * RW;                     // [kWarps][cap][NC] warp partials

    // (without particles the tile lists may not exist: only the faces kernel gets here then)
    const int cnt = (FACES && pd.n == 0) ? 0 : tl.count[tile];
    if (cnt == 0 && !FACES) return;                        // plain-fluid tile: k_fluid_pair does it
    const unsigned txy = tile / (unsigned)g.nt[0];          // 32-bit: tiles < 2^31 (host check)
    const int tx = (int)(tile - txy * (unsigned)g.nt[0]);
    const int ty = (int)(txy % (unsigned)g.nt[1]);
    const int tz = (int)(txy / (unsigned)g.nt[1]);
    const bool ovf = cnt > cap;
    const int nchunk = ovf ? (pd.n + cap - 1) / cap : 1;
    const T *recs = (FACES && cnt == 0) ? nullptr
                  : reinterpret_cast<const T *>(tl.blocks) + (size_t)tile * block_elems<T>(cap) + head_elems<T>();

    const int tid = threadIdx.x + L::TX * (threadIdx.y + L::TY * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5;
    const int x0 = tx * L::TX, y0 = ty * L::TY, z0 = tz * L::TZ;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    const bool active = cell_active<L>(g, x, y, z);
    const long long cell = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
    const long long N = g.ncell;

    // ---- 0. this thread's share of the tile's records (cap <= 64 records of RW values),
    //         loaded now, written to shared memory once the pull loads are in flight
    constexpr int kRecWords = (64 * RW + kThreads - 1) / kThreads;
    T rw[kRecWords];
    const int nwords = ovf ? 0 : cnt * RW;
#pragma unroll
    for (int j = 0; j < kRecWords; ++j) {
        const int w = tid + j * kThreads;
        rw[j] = (w < nwords) ? recs[w] : (T)0;
    }

    // ---- 1. pull (Eq. 1, Eq. 6)
    T df[Q];
    const bool interior = x0 >= 1 && x0 + L::TX < g.n[0] && y0 >= 1 && y0 + L::TY < g.n[1] &&
                          (L::D == 2 || (z0 >= 1 && z0 + L::TZ < g.n[2]));
    if (interior) {
        const S *base = fin + cell;
        const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            df[i] = Store<S>::ld(base, PSC_OFF(cell, (long long)i * N - (L::ex(i) + L::ey(i) * sy + L::ez(i) * sz), Q * N, CHK_POP), ph.sc);
    } else if (active) {
        if (FACES) {
            pull_all<L, S>(fin, g, x, y, z, cell, ph, df);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) df[i] = pull_one<L, S>(fin, g, x, y, z, cell, i, ph.sc);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) df[i] = (T)0;
    }

    // ---- 2. moments (Eq. 5): rho = 1 + sum d_i, rho u = j + F/2
    T drho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += df[i];
        if (L::ex(i)) jx += L::ex(i) * df[i];
        if (L::ey(i)) jy += L::ey(i) * df[i];
        if (L::ez(i)) jz += L::ez(i) * df[i];
    }
    const T rho = (T)1 + drho;
    const T irho = (T)1 / rho;
    const T ux = (jx + (T)0.5 * ph.F[0]) * irho;
    const T uy = (jy + (T)0.5 * ph.F[1]) * irho;
    const T uz = (jz + (T)0.5 * ph.F[2]) * irho;
    if (active && !(rho > (T)0)) atomicOr(flags, 1);

#pragma unroll
    for (int j = 0; j < kRecWords; ++j) {
        const int w = tid + j * kThreads;
        if (w < nwords) srec[w] = rw[j];
    }

    // ---- 3. candidates reaching this row: solid fractions and u_s moments of the cell
    const T cx = (T)threadIdx.x, cy = (T)threadIdx.y, cz = (T)threadIdx.z;
    const T xmax = (T)(min(L::TX, g.n[0] - x0) - 1);
    T seps = 0, mx = 0, my = 0, mz = 0, Mxx = 0, Myy = 0, Mzz = 0, Mxy = 0, Mxz = 0, Myz = 0;
    unsigned long long wmask = 0ull;     // relevant candidates of this row (normal tiles)
    T eslot[NSLOT] = {};                 // eps of the first relevant candidates, for step 6
    int nk = cnt;
    for (int ch = 0; ch < nchunk; ++ch) {
        if (ovf) {
            nk = min(cap, pd.n - ch * cap);
            __syncthreads();
            if (tid < nk) write_record<L, T>(srec + tid * RW, g, pd, ch * cap + tid, x0, y0, z0);
        }
        __syncthreads();
        int js = 0;
        for (int kb = 0; kb < nk; kb += 32) {
            const int k = kb + lane;
            bool rel = false;
            if (k < nk) {
                const Vec4<T> a = ld4<T>(srec + k * RW);
                rel = row_hits<L, T>(g, a.x, a.y, a.z, a.w + ph.h, cy, cz, xmax);
            }
            unsigned bal = __ballot_sync(kFull, rel);
            if (!ovf) wmask |= (unsigned long long)bal << kb;
            while (bal) {
                const int kk = kb + __ffs(bal) - 1;
                bal &= bal - 1u;
                const T *rk = srec + kk * RW;
                const Vec4<T> a = ld4<T>(rk);
                const Vec4<T> b = ld4<T>(rk + 4);      // f(r), Ux, Uy, Uz
                T dx, dy, dz;
                cand_arm<L, T>(g, cx, cy, cz, a.x, a.y, a.z, dx, dy, dz);
                const T e = active ? shell_eps<T>(dx * dx + dy * dy + dz * dz, a.w, b.x, ph.h) : (T)0;
                if (!ovf) {
#pragma unroll
                    for (int q = 0; q < NSLOT; ++q) if (js == q) eslot[q] = e;
                }
                ++js;
                if (e > (T)0) {
                    const Vec4<T> c = ld4<T>(rk + 8);  // Ox, Oy, Oz, id
                    // u_s = U + Omega x (x_n - X_p)
                    const T usx = b.y + c.y * dz - c.z * dy;
                    const T usy = b.z + c.z * dx - c.x * dz;
                    const T usz = (L::D == 3) ? b.w + c.x * dy - c.y * dx : (T)0;
                    // modified scheme weights by eps_s (normalised below); original by B(eps_s)
                    const T wgt = (PSC == 0) ? e : e * ph.tmh / (((T)1 - e) + ph.tmh);
                    seps += wgt;
                    mx += wgt * usx; my += wgt * usy; mz += wgt * usz;
                    Mxx += wgt * usx * usx; Myy += wgt * usy * usy; Mxy += wgt * usx * usy;
                    if (L::D == 3) { Mzz += wgt * usz * usz; Mxz += wgt * usx * usz; Myz += wgt * usy * usz; }
                }
            }
        }
    }

    // ---- 4. weights: eps_n = min(1, sum eps) (Table 1 Step 5), B_n by Eq. 9 at eps_n,
    //         B_{n,s} = B_n eps_s / sum eps = cB eps_s (Eq. 13; cells with overlapping
    //         fractions keep B_n = 1). Original scheme: B_n = sum_s B(eps_s) (Eq. 8).
    const bool any_solid = __any_sync(kFull, seps > (T)0);
    T Bn = 0, cB = 0;
    if (any_solid && seps > (T)0) {
        if (PSC == 0) {
            if (seps < (T)1) {
                const T c = ph.tmh / (((T)1 - seps) + ph.tmh);
                Bn = seps * c;
                cB = c;
            } else {
                Bn = (T)1;
                cB = (T)1 / seps;
            }
        } else {
            Bn = seps;
            cB = (T)1;
        }
        mx *= cB; my *= cB; mz *= cB;
        Mxx *= cB; Myy *= cB; Mzz *= cB; Mxy *= cB; Mxz *= cB; Myz *= cB;
    }

    // ---- 5. collision (Eq. 2-4, 10, 12) in deviation form, then store
    const T uu = ux * ux + uy * uy + uz * uz;
    const T uF = ux * ph.F[0] + uy * ph.F[1] + uz * ph.F[2];
    if (!any_solid) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T w = (T)weight<L>(i);
            const T eu = L::ex(i) * ux + L::ey(i) * uy + L::ez(i) * uz;
            const T eF = L::ex(i) * ph.F[0] + L::ey(i) * ph.F[1] + L::ez(i) * ph.F[2];
            const T dfeq = w * (drho + rho * ((T)3 * eu + (T)4.5 * eu * eu - (T)1.5 * uu));
            const T fi = ph.guo * w * ((T)3 * (eF - uF) + (T)9 * eu * eF);
            const T out = df[i] - ph.omega * (df[i] - dfeq) + fi;
            if (active) Store<S>::st(fout, PSC_IDX((long long)i * N + cell, Q * N, CHK_POP), out, ph.sc);
        }
    } else {
        const T trM = Mxx + Myy + Mzz;
        const T omB = (T)1 - Bn;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int o = opp<L>(i);
            const T w = (T)weight<L>(i);
            const T ex = (T)L::ex(i), ey = (T)L::ey(i), ez = (T)L::ez(i);
            const T eu = ex * ux + ey * uy + ez * uz;
            const T eF = ex * ph.F[0] + ey * ph.F[1] + ez * ph.F[2];
            const T sym = drho + rho * ((T)4.5 * eu * eu - (T)1.5 * uu);
            const T dfeq = w * (sym + rho * (T)3 * eu);
            const T dfeq_o = w * (sym - rho * (T)3 * eu);
            const T fi = ph.guo * w * ((T)3 * (eF - uF) + (T)9 * eu * eF);
            const T em = ex * mx + ey * my + ez * mz;
            const T eMe = ex * ex * Mxx + ey * ey * Myy + ez * ez * Mzz +
                          (T)2 * (ex * ey * Mxy + ex * ez * Mxz + ey * ez * Myz);
            const T sfe = w * (Bn * drho + rho * ((T)3 * em + (T)4.5 * eMe - (T)1.5 * trM));
            const T out = df[i] - omB * ph.omega * (df[i] - dfeq) + Bn * (df[o] - dfeq_o - df[i]) +
                          sfe + omB * fi;
            if (active) Store<S>::st(fout, PSC_IDX((long long)i * N + cell, Q * N, CHK_POP), out, ph.sc);
        }
    }

    // ---- 6. force and torque (Eq. 14; Eq. 11 in original mode):
    //         F_p -= B_{n,s} (rho u_s + F/2 - j),  T_p -= (x_n - X_p) x (same)
    const bool solid = active && seps > (T)0;
    const T px = (T)0.5 * ph.F[0] - jx, py = (T)0.5 * ph.F[1] - jy, pz = (T)0.5 * ph.F[2] - jz;
    if (!ovf && lane == 0) s_mask[warp] = any_solid ? wmask : 0ull;
    if (any_solid) {
        for (int ch = 0; ch < nchunk; ++ch) {
            if (ovf) {
                nk = min(cap, pd.n - ch * cap);
                __syncwarp();
                // overflow tiles: each warp restages nothing; records come from global memory
            }
            int js = 0;
            for (int kb = 0; kb < nk; kb += 32) {
                const int k = kb + lane;
                bool rel;
                T ovr[RW];
                if (!ovf) {
                    rel = (wmask >> k) & 1ull;
                } else {
                    rel = false;
                    if (k < nk) {
                        write_record<L, T>(ovr, g, pd, ch * cap + k, x0, y0, z0);
                        rel = row_hits<L, T>(g, ovr[R_PX], ovr[R_PY], ovr[R_PZ], ovr[R_R] + ph.h, cy, cz, xmax);
                    }
                }
                unsigned bal = __ballot_sync(kFull, rel);
                while (bal) {
                    const int src = __ffs(bal) - 1;
                    const int kk = kb + src;
                    bal &= bal - 1u;
                    T a[RW];
                    if (!ovf) {
#pragma unroll
                        for (int q = 0; q < RW; ++q) a[q] = srec[kk * RW + q];
                    } else {
#pragma unroll
                        for (int q = 0; q < RW; ++q) a[q] = __shfl_sync(kFull, ovr[q], src);
                    }
                    T v[NC];
#pragma unroll
                    for (int q = 0; q < NC; ++q) v[q] = (T)0;
                    if (solid) {
                        T dx, dy, dz;
                        cand_arm<L, T>(g, cx, cy, cz, a[R_PX], a[R_PY], a[R_PZ], dx, dy, dz);
                        T e = (T)0;
                        if (!ovf && js < NSLOT) {
#pragma unroll
                            for (int q = 0; q < NSLOT; ++q) if (js == q) e = eslot[q];
                        } else {
                            e = shell_eps<T>(dx * dx + dy * dy + dz * dz, a[R_R], a[R_FR], ph.h);
                        }
                        if (e > (T)0) {
                            const T usx = a[R_UX] + a[R_OY] * dz - a[R_OZ] * dy;
                            const T usy = a[R_UY] + a[R_OZ] * dx - a[R_OX] * dz;
                            const T usz = (L::D == 3) ? a[R_UZ] + a[R_OX] * dy - a[R_OY] * dx : (T)0;
                            const T Bs = (PSC == 0) ? cB * e : Bn;
                            const T dPx = Bs * (rho * usx + px);
                            const T dPy = Bs * (rho * usy + py);
                            const T dPz = (L::D == 3) ? Bs * (rho * usz + pz) : (T)0;
                            if (L::D == 2) {
                                v[0] = dPx; v[1] = dPy; v[2] = dx * dPy - dy * dPx;
                            } else {
                                v[0] = dPx; v[1] = dPy; v[2] = dPz;
                                v[3] = dy * dPz - dz * dPy;
                                v[4] = dz * dPx - dx * dPz;
                                v[5] = dx * dPy - dy * dPx;
                            }
                        }
                    }
                    ++js;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                        for (int q = 0; q < NC; ++q) v[q] += __shfl_xor_sync(kFull, v[q], off);
                    }
                    if (lane == 0) {
                        if (!ovf) {
#pragma unroll
                            for (int q = 0; q < NC; ++q) part[((size_t)warp * cap + kk) * NC + q] = v[q];
                        } else {
                            const int pid = (int)PSC_IDX(bits_id(a[R_ID]), pd.n, CHK_PART);
#pragma unroll
                            for (int q = 0; q < NC; ++q) {
                                if (v[q] == (T)0) continue;
                                double *dst;
                                if (L::D == 2) dst = (q < 2) ? &pd.F[3 * pid + q] : &pd.T[3 * pid + 2];
                                else dst = (q < 3) ? &pd.F[3 * pid + q] : &pd.T[3 * pid + q - 3];
                                atomicAdd(dst, -(double)v[q]);
                            }
                        }
                    }
                }
            }
        }
    }
    if (ovf) return;   // uniform over the block
    __syncthreads();
    // tile totals in a fixed warp order, one FP64 atomic per particle component
    for (int idx = tid; idx < cnt * NC; idx += kThreads) {
        const int k = idx / NC, q = idx - k * NC;
        T sum = 0;
        bool any = false;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            if ((s_mask[w] >> k) & 1ull) { sum += part[((size_t)w * cap + k) * NC + q]; any = true; }
        }
        if (any && sum != (T)0) {
            const int p = bits_id(srec[k * RW + R_ID]);
            double *dst;
            if (L::D == 2) dst = (q < 2) ? &pd.F[3 * p + q] : &pd.T[3 * p + 2];
            else dst = (q < 3) ? &pd.F[3 * p + q] : &pd.T[3 * p + q - 3];
            atomicAdd(dst, -(double)sum);
        }
    }
}

#include "psc_pair.cuh"

// Tiles with more candidates than the block holds (rare): the exact chunked path over all
// particles, one block per tile of the overflow list. With no such tile every block returns
// at once.
template <class L, typename S, int PSC>
__global__ void __launch_bounds__(kThreads, 1)
k_collide_overflow(const S *__restrict__ fin, S *__restrict__ fout, Geom g, PhysT<typename Store<S>::T> ph,
                   Tiles tl, Parts pd, int *flags) {
    using T = typename Store<S>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_mask[kWarps];
    const long long ntiles = (long long)g.nt[0] * g.nt[1] * g.nt[2];
    const int novf = tl.stats[2];
    // the collide-stream kernel before this one has finished: clear its work counters
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
        tl.stats[3] = 0;
        tl.stats[6] = 0;
    }
    for (int it = blockIdx.x; it < novf; it += gridDim.x) {
        psc_tile<L, S, PSC>(tl.order[2 * ntiles + it].x, fin, fout, g, ph, tl, pd, flags,
                            reinterpret_cast<T *>(smem), s_mask);
        __syncthreads();
    }
}

// Contexts with an open, inlet or outlet face: every tile, with or without candidates, by
// the single-cell path whose pull classifies each face (persistent blocks over the tiles).
template <class L, typename S, int PSC>
__global__ void __launch_bounds__(kThreads, 1)
k_collide_faces(const S *__restrict__ fin, S *__restrict__ fout, Geom g, PhysT<typename Store<S>::T> ph,
                Tiles tl, Parts pd, int *flags) {
    using T = typename Store<S>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_mask[kWarps];
    const long long ntiles = (long long)g.nt[0] * g.nt[1] * g.nt[2];
    for (long long it = blockIdx.x; it < ntiles; it += gridDim.x) {
        psc_tile<L, S, PSC, true>((unsigned)it, fin, fout, g, ph, tl, pd, flags,
                                  reinterpret_cast<T *>(smem), s_mask);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- gather / set kernels
template <class L, typename S>
__global__ void k_gather(const S *__restrict__ fin, Geom g, PhysT<typename Store<S>::T> ph,
                         double *f_out, double *rho_out, double *u_out) {
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= g.ncell) return;
    const int x = (int)(cell % g.n[0]);
    const int y = (int)((cell / g.n[0]) % g.n[1]);
    const int z = (int)(cell / ((long long)g.n[0] * g.n[1]));
    double drho = 0, j[3] = {0, 0, 0};
    typename Store<S>::T df[L::Q];
    pull_all<L, S>(fin, g, x, y, z, cell, ph, df);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const double d = (double)df[i];
        if (f_out) f_out[(long long)i * g.ncell + cell] = weight<L>(i) + d;
        drho += d;
        j[0] += L::ex(i) * d; j[1] += L::ey(i) * d; j[2] += L::ez(i) * d;
    }
    const double rho = 1.0 + drho;
    if (rho_out) rho_out[cell] = rho;
    if (u_out) {
        for (int a = 0; a < 3; ++a) u_out[3 * cell + a] = (j[a] + 0.5 * (double)ph.F[a]) / rho;
    }
}

// Inverse of the pull: the stored post-collision value f^+_i(x) is the pre-collision
// f_i(x + e_i), or f_{-i}(x) when x + e_i lies beyond a wall.
template <class L, typename S>
__global__ void k_set(const double *__restrict__ f, S *__restrict__ fout, Geom g,
                      PhysT<typename Store<S>::T> ph) {
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= g.ncell) return;
    const int xc[3] = {(int)(cell % g.n[0]), (int)((cell / g.n[0]) % g.n[1]),
                       (int)(cell / ((long long)g.n[0] * g.n[1]))};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
        int d[3];
        bool wall = false, leaves = false;
        for (int a = 0; a < 3; ++a) {
            d[a] = xc[a] + e[a];
            if (d[a] < 0 || d[a] >= g.n[a]) {
                const int kind = face_kind(g, a, d[a] < 0 ? 0 : 1);
                if (kind == FACE_PERIODIC) d[a] += (d[a] < 0) ? g.n[a] : -g.n[a];
                else if (kind == FACE_WALL) wall = true;
                else leaves = true;
            }
        }
        double v;
        if (wall) v = f[(long long)opp<L>(i) * g.ncell + cell];
        else if (leaves) v = f[(long long)i * g.ncell + cell];     // leaves the lattice: never pulled
        else v = f[(long long)i * g.ncell + d[0] + (long long)g.n[0] * (d[1] + (long long)g.n[1] * d[2])];
        Store<S>::st(fout, PSC_IDX((long long)i * g.ncell + cell, L::Q * g.ncell, CHK_POP), (typename Store<S>::T)(v - weight<L>(i)), ph.sc);
    }
}

// Blocks of a persistent grid: as many as stay resident on all SMs (never more than the
// work items). The occupancy query is cached per kernel and shared-memory size.
template <typename K>
inline cudaError_t persistent_blocks(K kern, size_t smem, long long work, unsigned &blocks, int threads = kThreads,
                                     int *per_sm = nullptr) {
    static thread_local const void *c_kern = nullptr;
    static thread_local size_t c_smem = (size_t)-1;
    static thread_local int c_per = 0;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (c_smem != smem || c_kern != (const void *)kern) {
        int per = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
        if (e != cudaSuccess) return e;
        c_per = per > 0 ? per : 1;
        c_smem = smem;
        c_kern = (const void *)kern;
    }
    const long long b = (long long)sms * c_per;
    blocks = (unsigned)(b < work ? b : (work > 0 ? work : 1));
    if (per_sm) *per_sm = c_per;
    return cudaSuccess;
}

// Registers a block of `threads` holds (allocated per warp in units of 8 per thread).
template <typename K>
inline cudaError_t block_registers(K kern, int threads, int &regs) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    regs = (e == cudaSuccess) ? ((fa.numRegs + 7) / 8 * 8) * threads : 0;
    return e;
}

// One collide-stream step. Without particles: the fluid kernel over every tile. With
// The overflow-tile kernel (tiles with more candidates than the pair kernels keep), which also
// clears the particle-tile kernel's work counters for the next launch.
template <class L, typename S, int PSC>
cudaError_t launch_overflow(const void *fin, void *fout, const Geom &g, const PhysT<typename Store<S>::T> &pt,
                            const Tiles &tl, const Parts &pd, int *flags, size_t osmem, dim3 block, cudaStream_t s) {
    auto okern = k_collide_overflow<L, S, PSC>;
    if (osmem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(okern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osmem);
        if (e != cudaSuccess) return e;
    }
    okern<<<32, block, osmem, s>>>((const S *)fin, (S *)fout, g, pt, tl, pd, flags);
    return cudaGetLastError();
}

// Fluid-tile blocks per SM when they follow the particle tiles beside the caller's next
// kernels (a deferred join). On the 2048^2 channel with 5000 discs and its DEM call the
// coupled step took 167.8 / 140.8 / 142.0 / 146.0 / 147.2 / 159.4 us with 1 / 2 / 3 / 4 / 5
// / 6 blocks per SM (156 us as two calls): fewer leave the fluid tiles unfinished when the
// DEM call ends, more slow the latency-bound DEM kernels down.
constexpr int kDeferF = 2;

// particles in 2D (FP32 and 16-bit storage): the particle-tile kernel (4 blocks per SM) and
// the fluid-tile kernel (3 blocks per SM) side by side on two streams, which together fill
// each SM's register file, so the issue-bound particle tiles and the DRAM-bound fluid tiles
// share every SM for the whole step; without a second stream, one after the other. In 3D
// (and FP64) the particle-tile kernel holds all the registers an SM has, and takes the
// fluid tiles itself once its own are done. Then the overflow kernel.
template <class L, typename S, int PSC>
cudaError_t launch_collide_stream_t(const void *fin, void *fout, const Geom &g, const Phys &ph,
                                    const Tiles &tl, const Parts &pd, int *flags, cudaStream_t s,
                                    Overlap *ov) {
    using T = typename Store<S>::T;
    constexpr int NC = (L::D == 2) ? 3 : 6;
    constexpr bool kSteal = (L::D == 3) || sizeof(T) == 8;
    // blocks per SM side by side (2D): 4 x 128 threads x 80 registers + 3 x 128 x 64 = 64 K
    constexpr int kSideP = 4, kSideF = 3;
    const size_t smem = pair_smem_bytes<L, T>();
    const size_t osmem = cs_smem_bytes<T>(tl.cap, NC);
    auto kern = k_collide_stream<L, S, PSC, kSteal>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long ntiles = (long long)g.nt[0] * g.nt[1] * g.nt[2];
    dim3 block(L::TX, L::TY, L::TZ);
    const PhysT<T> pt = make_phys<T>(ph, L::Q);
    bool faces = false;
    for (int a = 0; a < 3; ++a) faces |= face_kind(g, a, 0) >= FACE_OPEN || face_kind(g, a, 1) >= FACE_OPEN;
    if (faces) {
        auto fk = k_collide_faces<L, S, PSC>;
        if (osmem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osmem);
            if (e != cudaSuccess) return e;
        }
        unsigned nbf = 0;
        cudaError_t e = persistent_blocks(fk, osmem, ntiles, nbf, kThreads);
        if (e != cudaSuccess) return e;
        fk<<<nbf, block, osmem, s>>>((const S *)fin, (S *)fout, g, pt, tl, pd, flags);
        return cudaGetLastError();
    }
    const bool hasF = ph.body_force[0] != 0.0 || ph.body_force[1] != 0.0 || ph.body_force[2] != 0.0;
    auto fkern = hasF ? k_fluid_pair<L, S, true> : k_fluid_pair<L, S, false>;
    const dim3 pblock(32, kPWarps);
    if (pd.n == 0) {
        fkern<<<dim3(g.nt[0], g.nt[1], g.nt[2]), pblock, 0, s>>>((const S *)fin, (S *)fout, g, pt, tl, 0, flags);
        return cudaGetLastError();
    }
    cudaError_t e;
    unsigned nb = 0;
    bool side = false;
    int nsm = 0;
    if (!kSteal && ov && ov->aux) {
        int dev = 0, rf_sm = 0, rp = 0, rf = 0, per = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&rf_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        if (e == cudaSuccess) e = block_registers(kern, kPThreads, rp);
        if (e == cudaSuccess) e = block_registers(fkern, kPThreads, rf);
        if (e == cudaSuccess) e = persistent_blocks(kern, smem, ntiles, nb, kPThreads, &per);
        if (e != cudaSuccess) return e;
        side = per >= kSideP && kSideP * rp + kSideF * rf <= rf_sm;
    }
    if (side && ov->defer) {
        e = persistent_blocks(kern, smem, ntiles, nb, kPThreads);
        if (e != cudaSuccess) return e;
        kern<<<nb, pblock, smem, s>>>((const S *)fin, (S *)fout, g, pt, tl, pd, flags);
        e = launch_overflow<L, S, PSC>(fin, fout, g, pt, tl, pd, flags, osmem, block, s);
        if (e == cudaSuccess) e = cudaEventRecord(ov->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ov->aux, ov->fork, 0);
        if (e != cudaSuccess) return e;
        fkern<<<nsm * kDeferF, pblock, 0, ov->aux>>>((const S *)fin, (S *)fout, g, pt, tl, pd.n, flags);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ov->join, ov->aux);
        if (e == cudaSuccess) ov->deferred = 1;
        return e;
    }
    if (side) {
        e = cudaEventRecord(ov->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ov->aux, ov->fork, 0);
        if (e != cudaSuccess) return e;
        kern<<<nsm * kSideP, pblock, smem, s>>>((const S *)fin, (S *)fout, g, pt, tl, pd, flags);
        fkern<<<nsm * kSideF, pblock, 0, ov->aux>>>((const S *)fin, (S *)fout, g, pt, tl, pd.n, flags);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ov->join, ov->aux);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ov->join, 0);
        if (e != cudaSuccess) return e;
    } else {
        if (!kSteal) {
            e = persistent_blocks(fkern, 0, ntiles, nb, kPThreads);
            if (e != cudaSuccess) return e;
            fkern<<<nb, pblock, 0, s>>>((const S *)fin, (S *)fout, g, pt, tl, pd.n, flags);
        }
        e = persistent_blocks(kern, smem, ntiles, nb, kPThreads);
        if (e != cudaSuccess) return e;
        kern<<<nb, pblock, smem, s>>>((const S *)fin, (S *)fout, g, pt, tl, pd, flags);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_overflow<L, S, PSC>(fin, fout, g, pt, tl, pd, flags, osmem, block, s);
}

template <typename S>
cudaError_t launch_collide_stream_storage(int lattice, const void *fin, void *fout, const Geom &g,
                                          const Phys &ph, const Tiles &tl, const Parts &pd,
                                          int *flags, cudaStream_t s, Overlap *ov) {
    if (lattice == 9) {
        return ph.psc == 0 ? launch_collide_stream_t<D2Q9, S, 0>(fin, fout, g, ph, tl, pd, flags, s, ov)
                           : launch_collide_stream_t<D2Q9, S, 1>(fin, fout, g, ph, tl, pd, flags, s, ov);
    }
    return ph.psc == 0 ? launch_collide_stream_t<D3Q19, S, 0>(fin, fout, g, ph, tl, pd, flags, s, ov)
                       : launch_collide_stream_t<D3Q19, S, 1>(fin, fout, g, ph, tl, pd, flags, s, ov);
}

template <typename S>
cudaError_t launch_gather_storage(int lattice, const void *fin, double *f_out, double *rho,
                                  double *u, const Geom &g, const Phys &ph, cudaStream_t s) {
    using T = typename Store<S>::T;
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.ncell + threads - 1) / threads);
    if (lattice == 9) k_gather<D2Q9, S><<<blocks, threads, 0, s>>>((const S *)fin, g, make_phys<T>(ph, 9), f_out, rho, u);
    else k_gather<D3Q19, S><<<blocks, threads, 0, s>>>((const S *)fin, g, make_phys<T>(ph, 19), f_out, rho, u);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_set_storage(int lattice, const double *f, void *fout, const Geom &g,
                               const Phys &ph, cudaStream_t s) {
    using T = typename Store<S>::T;
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.ncell + threads - 1) / threads);
    if (lattice == 9) k_set<D2Q9, S><<<blocks, threads, 0, s>>>(f, (S *)fout, g, make_phys<T>(ph, 9));
    else k_set<D3Q19, S><<<blocks, threads, 0, s>>>(f, (S *)fout, g, make_phys<T>(ph, 19));
    return cudaGetLastError();
}

}  // namespace psc
