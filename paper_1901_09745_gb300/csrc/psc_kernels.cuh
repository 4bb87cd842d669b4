// psc_kernels.cuh -- sm_103a kernels of one lattice-Boltzmann step with the modified
// partially-saturated-cell (PSC) immersed moving boundary (Liu & Wu, arXiv 1901.09745).
//
// One thread block owns one lattice tile (32 x 8 cells in 2D, 32 x 4 x 2 in 3D), one thread
// per cell, x fastest so a warp reads 32 consecutive populations of one direction.
// Per step and cell the fused kernel
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
#include "psc_internal.h"

namespace psc {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct PhysT {
    T omega;        // 1/tau
    T tmh;          // tau - 1/2
    T guo;          // 1 - 1/(2 tau), Eq. 4
    T F[3];         // body force
    T h;            // Table 1 shell half-width
    float2 sc;      // (scale, 1/scale) of the stored deviations
};

template <typename T> __host__ PhysT<T> make_phys(const Phys &ph) {
    PhysT<T> k;
    k.omega = (T)(1.0 / ph.tau);
    k.tmh = (T)(ph.tau - 0.5);
    k.guo = (T)(1.0 - 1.0 / (2.0 * ph.tau));
    for (int a = 0; a < 3; ++a) k.F[a] = (T)ph.body_force[a];
    k.h = (T)ph.shell_h;
    k.sc = make_float2((float)ph.scale, (float)(1.0 / ph.scale));
    return k;
}

__device__ __forceinline__ float  rint_t(float v) { return rintf(v); }
__device__ __forceinline__ double rint_t(double v) { return rint(v); }
__device__ __forceinline__ float  sqrt_t(float v) { return sqrtf(v); }
__device__ __forceinline__ double sqrt_t(double v) { return sqrt(v); }

// Population i of cell (x, y, z) after streaming: the value the neighbour x - e_i stored
// in the previous step, or, when x - e_i lies beyond a wall, the value this cell stored in
// the opposite direction (halfway bounce-back, Eq. 6).
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
    if (bounce) return Store<S>::ld(fin, (long long)opp<L>(i) * g.ncell + cell, sc);
    long long src = (long long)s[0] + (long long)g.n[0] * ((long long)s[1] + (long long)g.n[1] * s[2]);
    return Store<S>::ld(fin, (long long)i * g.ncell + src, sc);
}

// Shared-memory candidate table of one tile: positions relative to the tile origin
// (minimum image), radius, f(r), velocity and spin, all in the compute type.
template <typename T> struct CandSmem {
    T *px, *py, *pz, *r, *fr, *ux, *uy, *uz, *ox, *oy, *oz;
    T *part;        // [kWarps][NC][cap] warp partial sums of force/torque
    int *id;        // [cap] particle index of each slot (sorted ascending)
    int *idraw;     // [cap] unsorted list as read from global memory
};

template <typename T>
__host__ __device__ inline size_t cand_smem_bytes(int cap, int nc) {
    return (size_t)cap * (11 + (size_t)kWarps * nc) * sizeof(T) + (size_t)cap * 2 * sizeof(int);
}

template <typename T>
__device__ __forceinline__ CandSmem<T> carve(unsigned char *smem, int cap, int nc) {
    CandSmem<T> c;
    T *p = reinterpret_cast<T *>(smem);
    c.px = p; c.py = p + cap; c.pz = p + 2 * cap; c.r = p + 3 * cap; c.fr = p + 4 * cap;
    c.ux = p + 5 * cap; c.uy = p + 6 * cap; c.uz = p + 7 * cap;
    c.ox = p + 8 * cap; c.oy = p + 9 * cap; c.oz = p + 10 * cap;
    c.part = p + 11 * cap;
    c.id = reinterpret_cast<int *>(c.part + (size_t)kWarps * nc * cap);
    c.idraw = c.id + cap;
    return c;
}

// Load one chunk of candidates into shared memory. Normal case: the tile's list, sorted by
// particle index (so the per-cell summation order does not depend on the binning's atomic
// order). Overflow case: particles [ch*cap, ch*cap + nk) of the global array.
template <class L, typename T>
__device__ void load_chunk(const CandSmem<T> &c, const Geom &g, const Tiles &tl, const Parts &pd,
                           long long tile, bool ovf, int ch, int nk, int x0, int y0, int z0,
                           int tid) {
    int pos = tid, id = 0;
    if (ovf) {
        id = ch * tl.cap + tid;
    } else {
        if (tid < nk) c.idraw[tid] = tl.list[tile * tl.cap + tid];
        __syncthreads();
        if (tid < nk) {
            id = c.idraw[tid];
            int rank = 0;
            for (int j = 0; j < nk; ++j) rank += (c.idraw[j] < id);
            pos = rank;
        }
    }
    if (tid < nk) {
        const int org[3] = {x0, y0, z0};
        const int ext[3] = {L::TX, L::TY, L::TZ};
        T rel[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a >= L::D) { rel[a] = (T)0; continue; }
            double d = pd.X[3 * id + a] - (double)org[a];
            if (g.periodic[a]) {
                // minimum image with respect to the tile centre
                double cen = 0.5 * (ext[a] - 1);
                double e = d - cen;
                e -= (double)g.n[a] * rint(e / (double)g.n[a]);
                d = e + cen;
            }
            rel[a] = (T)d;
        }
        c.px[pos] = rel[0]; c.py[pos] = rel[1]; c.pz[pos] = rel[2];
        c.r[pos] = (T)pd.R[id];
        c.fr[pos] = (T)pd.Fr[id];
        c.ux[pos] = (T)pd.U[3 * id + 0]; c.uy[pos] = (T)pd.U[3 * id + 1]; c.uz[pos] = (T)pd.U[3 * id + 2];
        c.ox[pos] = (T)pd.Om[3 * id + 0]; c.oy[pos] = (T)pd.Om[3 * id + 1]; c.oz[pos] = (T)pd.Om[3 * id + 2];
        c.id[pos] = id;
    }
}

// Solid fraction of candidate k at the cell with tile-relative centre (cx, cy, cz):
// Table 1 Steps 2-4 with the inside/outside branches as stated in Sec. 2.4 (distance
// <= r - h -> 1, >= r + h -> 0), else clamp(f(r) - D, 0, 1) with D = distance - r (Eq. 15).
// Returns 0 outside; on return (dx, dy, dz) is the arm x_n - X_p.
template <class L, typename T>
__device__ __forceinline__ T cand_eps(const CandSmem<T> &c, const Geom &g, int k, T cx, T cy, T cz,
                                      T h, T &dx, T &dy, T &dz) {
    dx = cx - c.px[k];
    dy = cy - c.py[k];
    dz = (L::D == 3) ? cz - c.pz[k] : (T)0;
    if (g.wrap_img[0]) dx -= (T)g.n[0] * rint_t(dx / (T)g.n[0]);
    if (g.wrap_img[1]) dy -= (T)g.n[1] * rint_t(dy / (T)g.n[1]);
    if (L::D == 3 && g.wrap_img[2]) dz -= (T)g.n[2] * rint_t(dz / (T)g.n[2]);
    const T d2 = dx * dx + dy * dy + dz * dz;
    const T r = c.r[k];
    const T rh = r + h;
    if (!(d2 < rh * rh)) return (T)0;
    const T dist = sqrt_t(d2);
    if (dist <= r - h) return (T)1;
    T e = c.fr[k] - (dist - r);
    e = e < (T)0 ? (T)0 : e;
    e = e > (T)1 ? (T)1 : e;
    return e;
}

template <class L, typename S, int PSC>
__global__ void __launch_bounds__(kThreads)
k_collide_stream(const S *__restrict__ fin, S *__restrict__ fout, Geom g,
                 PhysT<typename Store<S>::T> ph, Tiles tl, Parts pd, int *flags) {
    using T = typename Store<S>::T;
    constexpr int Q = L::Q;
    constexpr int NC = (L::D == 2) ? 3 : 6;
    extern __shared__ __align__(16) unsigned char smem[];
    const int cap = tl.cap;
    const CandSmem<T> c = carve<T>(smem, cap, NC);

    const int tid = threadIdx.x + L::TX * (threadIdx.y + L::TY * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5;
    const int x0 = blockIdx.x * L::TX, y0 = blockIdx.y * L::TY, z0 = blockIdx.z * L::TZ;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y, z = z0 + threadIdx.z;
    const bool active = x < g.n[0] && y < g.n[1] && z < g.n[2];
    const long long tile = blockIdx.x + (long long)g.nt[0] * (blockIdx.y + (long long)g.nt[1] * blockIdx.z);
    const long long cell = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
    const long long N = g.ncell;

    // ---- 1. pull (Eq. 1, Eq. 6)
    T df[Q];
    const bool interior = x0 >= 1 && x0 + L::TX < g.n[0] && y0 >= 1 && y0 + L::TY < g.n[1] &&
                          (L::D == 2 || (z0 >= 1 && z0 + L::TZ < g.n[2]));
    if (interior) {
        const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            df[i] = Store<S>::ld(fin, (long long)i * N + cell - (L::ex(i) + L::ey(i) * sy + L::ez(i) * sz), ph.sc);
    } else if (active) {
#pragma unroll
        for (int i = 0; i < Q; ++i) df[i] = pull_one<L, S>(fin, g, x, y, z, cell, i, ph.sc);
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

    // ---- 3. candidates: solid fractions and the u_s moments of the cell
    const int cnt = (pd.n > 0) ? tl.count[tile] : 0;
    const bool ovf = cnt > cap;
    const int nchunk = ovf ? (pd.n + cap - 1) / cap : (cnt > 0 ? 1 : 0);
    const T cx = (T)(x - x0), cy = (T)(y - y0), cz = (T)(z - z0);
    T seps = 0, mx = 0, my = 0, mz = 0, Mxx = 0, Myy = 0, Mzz = 0, Mxy = 0, Mxz = 0, Myz = 0;
    unsigned long long mask = 0ull;
    int nk = 0;
    for (int ch = 0; ch < nchunk; ++ch) {
        nk = ovf ? min(cap, pd.n - ch * cap) : cnt;
        __syncthreads();
        load_chunk<L, T>(c, g, tl, pd, tile, ovf, ch, nk, x0, y0, z0, tid);
        __syncthreads();
        if (!active) continue;
        for (int k = 0; k < nk; ++k) {
            T dx, dy, dz;
            const T e = cand_eps<L, T>(c, g, k, cx, cy, cz, ph.h, dx, dy, dz);
            if (e > (T)0) {
                // u_s = U + Omega x (x_n - X_p)
                const T usx = c.ux[k] + c.oy[k] * dz - c.oz[k] * dy;
                const T usy = c.uy[k] + c.oz[k] * dx - c.ox[k] * dz;
                const T usz = (L::D == 3) ? c.uz[k] + c.ox[k] * dy - c.oy[k] * dx : (T)0;
                // modified scheme weights by eps_s (normalised below); original by B(eps_s)
                const T wgt = (PSC == 0) ? e : e * ph.tmh / (((T)1 - e) + ph.tmh);
                seps += wgt;
                mx += wgt * usx; my += wgt * usy; mz += wgt * usz;
                Mxx += wgt * usx * usx; Myy += wgt * usy * usy; Mxy += wgt * usx * usy;
                if (L::D == 3) { Mzz += wgt * usz * usz; Mxz += wgt * usx * usz; Myz += wgt * usy * usz; }
                if (!ovf) mask |= (1ull << k);
            }
        }
    }

    // ---- 4. weights: eps_n = min(1, sum eps) (Table 1 Step 5), B_n by Eq. 9 at eps_n,
    //         B_{n,s} = B_n eps_s / sum eps (Eq. 13; bounded by one when fractions overlap)
    T Bn, cB;
    if (PSC == 0) {
        const T en = seps < (T)1 ? seps : (T)1;
        Bn = en * ph.tmh / (((T)1 - en) + ph.tmh);
        cB = seps > (T)0 ? Bn / seps : (T)0;
    } else {
        Bn = seps;    // Eq. 8: B_n = sum_s B(eps_s)
        cB = (T)1;
    }
    mx *= cB; my *= cB; mz *= cB;
    Mxx *= cB; Myy *= cB; Mzz *= cB; Mxy *= cB; Mxz *= cB; Myz *= cB;

    // ---- 5. collision (Eq. 2-4, 10, 12) in deviation form, then store
    const T uu = ux * ux + uy * uy + uz * uz;
    const T uF = ux * ph.F[0] + uy * ph.F[1] + uz * ph.F[2];
    const bool any_solid = __any_sync(kFull, Bn > (T)0);
    if (!any_solid) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T w = (T)weight<L>(i);
            const T eu = L::ex(i) * ux + L::ey(i) * uy + L::ez(i) * uz;
            const T eF = L::ex(i) * ph.F[0] + L::ey(i) * ph.F[1] + L::ez(i) * ph.F[2];
            const T dfeq = w * (drho + rho * ((T)3 * eu + (T)4.5 * eu * eu - (T)1.5 * uu));
            const T fi = ph.guo * w * ((T)3 * (eF - uF) + (T)9 * eu * eF);
            const T out = df[i] - ph.omega * (df[i] - dfeq) + fi;
            if (active) Store<S>::st(fout, (long long)i * N + cell, out, ph.sc);
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
            if (active) Store<S>::st(fout, (long long)i * N + cell, out, ph.sc);
        }
    }

    // ---- 6. force and torque (Eq. 14; Eq. 11 in original mode):
    //         F_p -= B_{n,s} (rho u_s + F/2 - j),  T_p -= (x_n - X_p) x (same)
    const bool touched = __syncthreads_or(seps > (T)0);
    if (!touched) return;
    const T px = (T)0.5 * ph.F[0] - jx, py = (T)0.5 * ph.F[1] - jy, pz = (T)0.5 * ph.F[2] - jz;
    for (int ch = 0; ch < nchunk; ++ch) {
        if (nchunk > 1) {
            nk = ovf ? min(cap, pd.n - ch * cap) : cnt;
            __syncthreads();
            load_chunk<L, T>(c, g, tl, pd, tile, ovf, ch, nk, x0, y0, z0, tid);
            __syncthreads();
        }
        for (int k = 0; k < nk; ++k) {
            const bool has = active && (ovf || ((mask >> k) & 1ull));
            T v[NC];
#pragma unroll
            for (int q = 0; q < NC; ++q) v[q] = (T)0;
            bool hit = false;
            if (has) {
                T dx, dy, dz;
                const T e = cand_eps<L, T>(c, g, k, cx, cy, cz, ph.h, dx, dy, dz);
                if (e > (T)0) {
                    hit = true;
                    const T usx = c.ux[k] + c.oy[k] * dz - c.oz[k] * dy;
                    const T usy = c.uy[k] + c.oz[k] * dx - c.ox[k] * dz;
                    const T usz = (L::D == 3) ? c.uz[k] + c.ox[k] * dy - c.oy[k] * dx : (T)0;
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
            const unsigned b = __ballot_sync(kFull, hit);
            if (b != 0u) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
                    for (int q = 0; q < NC; ++q) v[q] += __shfl_xor_sync(kFull, v[q], off);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int q = 0; q < NC; ++q) c.part[((size_t)warp * NC + q) * cap + k] = (b != 0u) ? v[q] : (T)0;
            }
        }
        __syncthreads();
        for (int idx = tid; idx < nk * NC; idx += kThreads) {
            const int k = idx / NC, q = idx - k * NC;
            T s = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s += c.part[((size_t)w * NC + q) * cap + k];
            if (s != (T)0) {
                const int p = c.id[k];
                double *dst;
                if (L::D == 2) dst = (q < 2) ? &pd.F[3 * p + q] : &pd.T[3 * p + 2];
                else dst = (q < 3) ? &pd.F[3 * p + q] : &pd.T[3 * p + q - 3];
                atomicAdd(dst, -(double)s);
            }
        }
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
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const double d = (double)pull_one<L, S>(fin, g, x, y, z, cell, i, ph.sc);
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
        bool wall = false;
        for (int a = 0; a < 3; ++a) {
            d[a] = xc[a] + e[a];
            if (d[a] < 0 || d[a] >= g.n[a]) {
                if (g.periodic[a]) d[a] += (d[a] < 0) ? g.n[a] : -g.n[a];
                else wall = true;
            }
        }
        double v;
        if (wall) v = f[(long long)opp<L>(i) * g.ncell + cell];
        else v = f[(long long)i * g.ncell + d[0] + (long long)g.n[0] * (d[1] + (long long)g.n[1] * d[2])];
        Store<S>::st(fout, (long long)i * g.ncell + cell, (typename Store<S>::T)(v - weight<L>(i)), ph.sc);
    }
}

template <class L, typename S, int PSC>
cudaError_t launch_collide_stream_t(const void *fin, void *fout, const Geom &g, const Phys &ph,
                                    const Tiles &tl, const Parts &pd, int *flags, cudaStream_t s) {
    using T = typename Store<S>::T;
    constexpr int NC = (L::D == 2) ? 3 : 6;
    const size_t smem = cand_smem_bytes<T>(tl.cap, NC);
    auto kern = k_collide_stream<L, S, PSC>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(g.nt[0], g.nt[1], g.nt[2]);
    dim3 block(L::TX, L::TY, L::TZ);
    kern<<<grid, block, smem, s>>>((const S *)fin, (S *)fout, g, make_phys<T>(ph), tl, pd, flags);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_collide_stream_storage(int lattice, const void *fin, void *fout, const Geom &g,
                                          const Phys &ph, const Tiles &tl, const Parts &pd,
                                          int *flags, cudaStream_t s) {
    if (lattice == 9) {
        return ph.psc == 0 ? launch_collide_stream_t<D2Q9, S, 0>(fin, fout, g, ph, tl, pd, flags, s)
                           : launch_collide_stream_t<D2Q9, S, 1>(fin, fout, g, ph, tl, pd, flags, s);
    }
    return ph.psc == 0 ? launch_collide_stream_t<D3Q19, S, 0>(fin, fout, g, ph, tl, pd, flags, s)
                       : launch_collide_stream_t<D3Q19, S, 1>(fin, fout, g, ph, tl, pd, flags, s);
}

template <typename S>
cudaError_t launch_gather_storage(int lattice, const void *fin, double *f_out, double *rho,
                                  double *u, const Geom &g, const Phys &ph, cudaStream_t s) {
    using T = typename Store<S>::T;
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.ncell + threads - 1) / threads);
    if (lattice == 9) k_gather<D2Q9, S><<<blocks, threads, 0, s>>>((const S *)fin, g, make_phys<T>(ph), f_out, rho, u);
    else k_gather<D3Q19, S><<<blocks, threads, 0, s>>>((const S *)fin, g, make_phys<T>(ph), f_out, rho, u);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_set_storage(int lattice, const double *f, void *fout, const Geom &g,
                               const Phys &ph, cudaStream_t s) {
    using T = typename Store<S>::T;
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.ncell + threads - 1) / threads);
    if (lattice == 9) k_set<D2Q9, S><<<blocks, threads, 0, s>>>(f, (S *)fout, g, make_phys<T>(ph));
    else k_set<D3Q19, S><<<blocks, threads, 0, s>>>(f, (S *)fout, g, make_phys<T>(ph));
    return cudaGetLastError();
}

}  // namespace psc
