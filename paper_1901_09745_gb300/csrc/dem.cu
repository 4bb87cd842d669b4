// dem.cu -- adhesive DEM contact update on the GPU (Liu & Wu, arXiv 1901.09745, Sec. 2.5).
//
// Per dem_step call (one LBM step):
//   0. k_dem_decide: whether the neighbour list is rebuilt in this call: when a sub-step
//                  of the previous call saw a particle a quarter of the skin away from
//                  where it was at the last build, or the host changed the particles.
//   1. k_dem_bin:  FP32 copies of the positions and velocities; on a rebuild, particles
//                  into a uniform bin grid (bin side >= 2 r_max + skin).
//   2. k_dem_nbr:  on a rebuild, one warp per particle builds its neighbour list (every j
//                  with |X_j - X_i| < r_i + r_j + skin), sorted by j, into the other of the
//                  two list buffers, carrying each pair's contact history over from the
//                  current one. Between rebuilds the sub-steps keep the current list: a
//                  pair not on it was farther apart than r_i + r_j + skin at the build, and
//                  neither particle has moved skin/2 since (a sub-step that sees one move
//                  that far reports it), so it cannot touch.
//   3. k_dem_substep (x substeps): two lanes per particle, each taking every other
//                  neighbour slot:
//        contact detection in FP64 with IEEE-rounded operations only (no FMA), so both
//        ends of a pair and a CPU reference agree bit for bit on delta_N;
//        the contact law in FP32: JKR normal force (Eq. 26-27) with the contact radius
//        from a bounded Newton solve, damping, sliding / twisting / rolling
//        spring-dashpot-sliders capped at Eq. 29, assembly of Eq. 22;
//        per-particle sums in FP64 (warp shuffles) and semi-implicit Euler in FP64
//        (Eq. 21) with the hydrodynamic force and torque of the last LBM step held fixed
//        over the sub-steps.
// Every pair is evaluated by both of its particles (each keeps its own copy of the pair's
// history); the two views are exact negations of each other, so no atomics are needed and
// the result does not depend on scheduling.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "capi_internal.h"
#include "hostdev.cuh"

namespace {

using psc::axis_at;
using psc::axis_span;
using psc::contact_sign;
using psc::ContactSign;
using psc::jkr_s;
using psc::moved2;

constexpr int kNB = 32;        // neighbour slots per particle (one warp lane each)
constexpr int kH = 8;          // history floats per slot: xi_s[3], xi_t, xi_r[3], contact flag
static_assert(kH == 8, "history slots are copied as two float4");
constexpr unsigned kFullMask = 0xffffffffu;
constexpr double kPi = 3.14159265358979323846;

struct DemGeom {
    int dim;
    int n[3];
    int periodic[3];
    int nb[3];          // bins per axis
    int bin_cap;
    double skin;
    float margin;       // slack for FP32 position copies (>> their rounding error)
    double inv_n[3];    // 1 / n per axis (no FP64 division on the device)
    double bscale[3];   // nb / n per axis: bin of x = floor(x * bscale)
};

struct DemPhys {
    float Es;           // effective modulus E* of Eq. 25 (one material)
    float Gs;           // effective shear modulus G*
    float gamma, mu_f, theta_crit, alpha_n, kt_scale, etat_scale;
    double dt, density;
    double g[3];
    int adhesive;
    double dc_coef;     // 1 / (2 cbrt(6)) for delta_C = a0^2 / (2 cbrt(6) R)
};

struct DemBufs {
    int n;
    const double *X, *U, *Om, *R;   // state at the start of the sub-step
    const float4 *Xf;               // FP32 copy (x, y, z, r) of the same positions
    float4 *Xfo;                    // FP32 copy of the new positions
    const float4 *Vf;               // FP32 copy of U, Omega: [n][2] {Ux, Uy, Uz, Ox}, {Oy, Oz, 0, 0}
    float4 *Vfo;                    // the same of the new velocities
    double *Xo, *Uo, *Omo;          // state at its end
    const double *Ff, *Tf;          // hydrodynamic force / torque (frozen)
    const double *Xref;             // positions when the neighbour list was built
    const int *nbr_n[2], *nbr[2];   // neighbour counts and slots [n][kNB] of both lists
    float *hist[2];                 // [n][kNB][kH] of both lists
    int *state;                     // DemState words (the current list is state[kListIdx])
    float *whist;                   // [n][3][kH] history of each particle's wall contacts, per axis
    const double *minv;             // [n][2]: 1/m, 1/I
    int *flags;                     // [1] solve failures, [2] list overflow, [3] skin exceeded
    float reject;                   // pairs with an FP32 overlap below -reject cannot touch
};

// Device words of a DEM context: a rebuild request (nonzero: rebuild the neighbour list at
// the next call; set by a sub-step, a particle upload or the host), the index (0/1) of the
// current list buffer, this call's decision, and the number of rebuilds so far.
enum { kRebuildReq = 0, kListIdx = 1, kRebuildNow = 2, kRebuilds = 3, kStateWords = 4 };

// Programmatic dependent launch: a kernel launched with that attribute may start while the
// kernel before it in the stream runs; it waits here until that kernel has finished and its
// writes are visible, before touching anything the predecessor produced. A kernel lets its
// successor start early with dep_launch().
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The call's decision (thread 0), and the bin counts cleared for the binning (all threads;
// unused when the list is kept).
__global__ void k_dem_decide(int *state, int *count, long long nbins) {
    dep_wait();
    dep_launch();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long k = t; k < nbins; k += (long long)gridDim.x * blockDim.x) count[k] = 0;
    if (t == 0) {
        const int rb = state[kRebuildReq] != 0;
        state[kRebuildNow] = rb;
        if (rb) { state[kListIdx] ^= 1; state[kRebuilds] += 1; }
        state[kRebuildReq] = 0;
    }
}

__device__ __forceinline__ int bin_of(double x, double bscale, int nb, int periodic) {
    int b = (int)floor(x * bscale);
    if (periodic) { b %= nb; if (b < 0) b += nb; }
    else { b = b < 0 ? 0 : (b >= nb ? nb - 1 : b); }
    return b;
}

__global__ void k_dem_bin(DemGeom g, int n, const double *X, const double *R, const double *U,
                          const double *Om, float4 *Xf, float4 *Vf, int *count, int *list, int *flags,
                          const int *state) {
    dep_wait();
    dep_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Xf[i] = make_float4((float)X[3 * i], (float)X[3 * i + 1], (float)X[3 * i + 2], (float)R[i]);
    Vf[2 * i] = make_float4((float)U[3 * i], (float)U[3 * i + 1], (float)U[3 * i + 2], (float)Om[3 * i]);
    Vf[2 * i + 1] = make_float4((float)Om[3 * i + 1], (float)Om[3 * i + 2], 0.0f, 0.0f);
    if (!state[kRebuildNow]) return;
    int b[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (a < g.dim) b[a] = bin_of(X[3 * i + a], g.bscale[a], g.nb[a], g.periodic[a]);
    const int bin = b[0] + g.nb[0] * (b[1] + g.nb[1] * b[2]);
    const int slot = atomicAdd(&count[bin], 1);
    if (slot < g.bin_cap) list[bin * g.bin_cap + slot] = i;
    else atomicAdd(&flags[2], 1);
}

__device__ __forceinline__ void mass_inertia(int dim, double rho, double r, double *m, double *I);

__global__ void k_dem_nbr(DemGeom g, int n, const double *X, const double *R, const float4 *Xf,
                          const int *count, const int *list, int *const *lists_n, int *const *lists,
                          float *const *hists, double *Xref, double *minv, double density, int *flags,
                          const int *state) {
    __shared__ int s_buf[8][kNB];
    dep_wait();
    dep_launch();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= n || !state[kRebuildNow]) return;   // whole warp leaves together
    // the new list goes to the buffer the decision selected; the previous one is the other
    const int nw = state[kListIdx], od = nw ^ 1;
    const int *old_n = lists_n[od], *old_nbr = lists[od];
    const float *old_hist = hists[od];
    int *new_n = lists_n[nw], *new_nbr = lists[nw];
    float *new_hist = hists[nw];
    const double xi[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
    const double ri = R[i];
    const float4 pi = Xf[i];
    // the previous list of i, one slot per lane (for the history carry-over below)
    const int on = old_n[i];
    const int oldj = (lane < on) ? old_nbr[i * kNB + lane] : -1;
    double mi = 0.0, ii = 0.0;
    if (lane == 0) {
        double m, I;
        mass_inertia(g.dim, density, ri, &m, &I);
        mi = 1.0 / m;
        ii = 1.0 / I;
    }
    int sx, sy, sz = 0, nbx, nby, nbz = 1;
    axis_span(bin_of(xi[0], g.bscale[0], g.nb[0], g.periodic[0]), g.nb[0], g.periodic[0], sx, nbx);
    axis_span(bin_of(xi[1], g.bscale[1], g.nb[1], g.periodic[1]), g.nb[1], g.periodic[1], sy, nby);
    if (g.dim == 3) axis_span(bin_of(xi[2], g.bscale[2], g.nb[2], g.periodic[2]), g.nb[2], g.periodic[2], sz, nbz);
    // the (up to 27) neighbouring bins: lane b holds bin b and its slot count, then a warp
    // prefix sum lets the lanes walk all slots of all bins 32 at a time
    const int nbins = nbx * nby * nbz;
    int mybin = 0, mycnt = 0;
    if (lane < nbins) {
        const int c = lane % nbx, bb = (lane / nbx) % nby, aa = lane / (nbx * nby);
        const int cz = (g.dim == 3) ? axis_at(aa, sz, g.nb[2], g.periodic[2]) : 0;
        mybin = axis_at(c, sx, g.nb[0], g.periodic[0]) + g.nb[0] * (axis_at(bb, sy, g.nb[1], g.periodic[1]) + g.nb[1] * cz);
        mycnt = min(count[mybin], g.bin_cap);
    }
    int incl = mycnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(kFullMask, incl, off);
        if (lane >= off) incl += v;
    }
    const int total = __shfl_sync(kFullMask, incl, 31);
    const int excl = incl - mycnt;
    const float reach0 = (float)ri + (float)g.skin + g.margin;
    int cnt = 0;
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        // which bin holds slot t: the last bin whose exclusive prefix is <= t (all lanes
        // take part in the shuffles; lanes past the end use the last slot and discard it)
        const int tc = min(t, total - 1);
        int owner = 0;
        for (int q = 0; q < nbins; ++q) {
            const int eq = __shfl_sync(kFullMask, excl, q);
            owner = (eq <= tc) ? q : owner;
        }
        const int ob = __shfl_sync(kFullMask, mybin, owner);
        const int oe = __shfl_sync(kFullMask, excl, owner);
        bool take = false;
        int j = -1;
        if (t < total) {
            j = list[ob * g.bin_cap + (t - oe)];
            if (j != i) {
                const float4 pj = Xf[j];
                float d2 = 0.0f;
                const float dd[3] = {pj.x - pi.x, pj.y - pi.y, pj.z - pi.z};
#pragma unroll
                for (int ax = 0; ax < 3; ++ax) {
                    if (ax >= g.dim) break;
                    float d = dd[ax];
                    if (g.periodic[ax]) {
                        const float half = 0.5f * (float)g.n[ax];
                        if (d > half) d -= (float)g.n[ax];
                        else if (d < -half) d += (float)g.n[ax];
                    }
                    d2 += d * d;
                }
                const float reach = reach0 + pj.w;
                take = d2 < reach * reach;
            }
        }
        const unsigned bal = __ballot_sync(kFullMask, take);
        const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
        if (take && pos < kNB) s_buf[warp][pos] = j;
        cnt += __popc(bal);
    }
    if (cnt > kNB) { if (lane == 0) atomicAdd(&flags[2], 1); cnt = kNB; }
    __syncwarp();
    // sort the slots by neighbour index (rank sort within the warp)
    int j = (lane < cnt) ? s_buf[warp][lane] : 0x7fffffff;
    int rank = 0;
    for (int q = 0; q < cnt; ++q) rank += (s_buf[warp][q] < j);
    __syncwarp();
    if (lane < cnt) s_buf[warp][rank] = j;
    __syncwarp();
    j = (lane < cnt) ? s_buf[warp][lane] : -2;
    // carry each pair's history over from the previous list of i: the slot whose neighbour
    // is j (lists hold each neighbour once)
    int found = -1;
    for (int q = 0; q < on; ++q) {
        const int v = __shfl_sync(kFullMask, oldj, q);
        if (v == j) found = q;
    }
    if (lane < cnt) {
        new_nbr[i * kNB + lane] = j;
        float4 *dst = reinterpret_cast<float4 *>(new_hist + ((size_t)i * kNB + lane) * kH);
        if (found >= 0) {
            const float4 *src = reinterpret_cast<const float4 *>(old_hist + ((size_t)i * kNB + found) * kH);
            dst[0] = src[0];
            dst[1] = src[1];
        } else {
            dst[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            dst[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    if (lane == 0) {
        new_n[i] = cnt;
        for (int a = 0; a < 3; ++a) Xref[3 * i + a] = xi[a];
        minv[2 * i] = mi;
        minv[2 * i + 1] = ii;
    }
}

__device__ __forceinline__ void cross3f(const float *a, const float *b, float *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float dot3f(const float *a, const float *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

__device__ __forceinline__ void rotate_into_plane(float *xi, const float *n) {
    const float len0 = sqrtf(dot3f(xi, xi));
    const float dn = dot3f(xi, n);
    for (int a = 0; a < 3; ++a) xi[a] -= dn * n[a];
    const float len1 = sqrtf(dot3f(xi, xi));
    if (len1 > 0.0f) { const float s = len0 / len1; for (int a = 0; a < 3; ++a) xi[a] *= s; }
}

// One contact seen from particle i (neighbour j): force and torque on i in FP32. The caller
// has decided whether the pair is in contact (exactly, see k_dem_substep) and passes the
// unit normal n (from i towards j) and the overlap delta_N in FP32. hist is this view's copy
// of the pair history; returns 0 and clears it when not in contact.
// Rf and ms are the contact's effective radius and mass (Eq. 25: 1/R = 1/r_i + 1/r_j,
// m* = m_i m_j / (m_i + m_j); against a wall R = r_i, m* = m_i, and rjf = 0 puts j's contact
// point on the wall, which does not move).
__device__ bool contact_on_i(const DemPhys &ph, int dim, const bool contact, const float *n, const float dnf,
                             const float rif, const float rjf, const float Rf, const float ms, const float *Ui,
                             const float *Uj, const float *omi, const float *omj, float *h,
                             float *fo, float *to, int *fail) {
    const float Es = ph.Es;
    float FC = 0.0f, a0 = 0.0f;
    if (ph.adhesive) {
        FC = (float)(3.0 * kPi) * ph.gamma * Rf;
        a0 = cbrtf((float)(9.0 * kPi) * ph.gamma * Rf * Rf / Es);
    }
    if (!contact) {
        for (int k = 0; k < kH; ++k) h[k] = 0.0f;
        for (int a = 0; a < 3; ++a) { fo[a] = 0.0f; to[a] = 0.0f; }
        return false;
    }
    float ac, Fne, kr = 0.0f, s_store = 1.0f;
    if (ph.adhesive) {
        const float s = jkr_s(dnf * Rf / (a0 * a0), fail, h[7]);
        s_store = s;
        const float s3 = s * s * s;
        ac = s * s * a0;
        Fne = 4.0f * FC * (s3 * s3 - s3);          // Eq. 26 with (a/a0)^3 = s^6, (a/a0)^1.5 = s^3
        kr = 4.0f * FC * s3;
    } else {
        const float dp = fmaxf(dnf, 0.0f);
        ac = sqrtf(Rf * dp);
        Fne = (4.0f / 3.0f) * Es * sqrtf(Rf) * dp * sqrtf(dp);
    }
    const float kN = 2.0f * Es * ac;
    const float etaN = ph.alpha_n * sqrtf(ms * kN);
    const float kT = ph.kt_scale * 8.0f * ph.Gs * ac;
    const float etaT = ph.etat_scale * etaN;
    const float dt = (float)ph.dt;

    // relative velocity of the contact points
    const float arm_i[3] = {rif * n[0], rif * n[1], rif * n[2]};
    const float arm_j[3] = {-rjf * n[0], -rjf * n[1], -rjf * n[2]};
    float w1[3], w2[3], vij[3], vt[3];
    cross3f(omi, arm_i, w1);
    cross3f(omj, arm_j, w2);
    for (int a = 0; a < 3; ++a) vij[a] = (Ui[a] + w1[a]) - (Uj[a] + w2[a]);
    const float vn = dot3f(vij, n);
    for (int a = 0; a < 3; ++a) vt[a] = vij[a] - vn * n[a];

    const float Fn = Fne + etaN * vn;

    // sliding
    const float Fscrit = ph.mu_f * fabsf(Fne + 2.0f * FC);
    float *xs = h, *xr = h + 4;
    rotate_into_plane(xs, n);
    for (int a = 0; a < 3; ++a) xs[a] += vt[a] * dt;
    float Ft[3];
    for (int a = 0; a < 3; ++a) Ft[a] = -kT * xs[a] - etaT * vt[a];
    float mag = sqrtf(dot3f(Ft, Ft));
    if (mag > Fscrit) {
        const float sc = Fscrit / mag;
        for (int a = 0; a < 3; ++a) Ft[a] *= sc;
        if (kT > 0.0f) for (int a = 0; a < 3; ++a) xs[a] = -Ft[a] / kT;
    }

    // twisting
    const float omrel[3] = {omi[0] - omj[0], omi[1] - omj[1], omi[2] - omj[2]};
    const float Omt = dot3f(omrel, n);
    h[3] += Omt * dt;
    float Mt = -(kT * ac * ac * 0.5f) * h[3] - (etaT * ac * ac * 0.5f) * Omt;
    const float Mtcrit = (float)(3.0 * kPi / 16.0) * ac * Fscrit;
    if (fabsf(Mt) > Mtcrit) {
        Mt = (Mt > 0.0f ? 1.0f : -1.0f) * Mtcrit;
        if (kT * ac * ac > 0.0f) h[3] = -Mt / (kT * ac * ac * 0.5f);
    }

    // rolling
    float Mr[3] = {0.0f, 0.0f, 0.0f};
    if (ph.adhesive) {
        const float Mrcrit = kr * ph.theta_crit * Rf;
        float vL[3], t[3];
        rotate_into_plane(xr, n);
        cross3f(n, omrel, vL);
        for (int a = 0; a < 3; ++a) xr[a] += Rf * vL[a] * dt;
        cross3f(n, xr, t);
        for (int a = 0; a < 3; ++a) Mr[a] = kr * t[a];
        mag = sqrtf(dot3f(Mr, Mr));
        if (mag > Mrcrit) {
            const float sc = Mrcrit / mag;
            for (int a = 0; a < 3; ++a) { Mr[a] *= sc; xr[a] *= sc; }
        }
    }
    h[7] = s_store;     // contact flag; JKR: the contact-radius root s (> 0)

    float tq[3];
    cross3f(arm_i, Ft, tq);
    for (int a = 0; a < 3; ++a) {
        fo[a] = -Fn * n[a] + Ft[a];
        to[a] = tq[a] + Mt * n[a] + Mr[a];
    }
    if (dim == 2) { fo[2] = 0.0f; to[0] = 0.0f; to[1] = 0.0f; }
    return true;
}

__device__ __forceinline__ void mass_inertia(int dim, double rho, double r, double *m, double *I) {
    if (dim == 2) { *m = rho * kPi * r * r; *I = 0.5 * (*m) * r * r; }
    else { *m = rho * (4.0 / 3.0) * kPi * r * r * r; *I = 0.4 * (*m) * r * r; }
}

constexpr int kLPP = 2;   // lanes per particle in the sub-step kernel (c2 coupled step: 1 lane
                          // 182.9 us, 2 lanes 162.0, 4 lanes 170.2, 8 lanes 206.0)

// One DEM sub-step. kLPP lanes share a particle and split its neighbour slots; their FP64
// sums are combined with shuffles in a fixed order, then the first lane integrates.
// early = 1 when the kernel before it in the stream is the previous sub-step of the same call.
template <int DIM>
__global__ void k_dem_substep(DemGeom g, DemPhys ph, DemBufs b, int early) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / kLPP, sub = t % kLPP;
    const bool valid = i < b.n;
    constexpr int dim = DIM;
    // Values fixed over a call's sub-steps: the list in use, the particle's neighbour count
    // and first neighbour, its radius and masses, the fluid's F and T (read by the
    // integrating lane before the contact loop's stores) and the position at the list's
    // build. After a sub-step of the same call they are loaded before waiting for it, so
    // the wait leads straight to the loads of the state that sub-step wrote.
    int li = 0, nn = 0, jn = 0;
    double ri = 1.0, fi[3] = {0, 0, 0}, ti[3] = {0, 0, 0}, xr[3] = {0, 0, 0}, im = 0.0, iI = 0.0;
    float imi = 0.0f;
    auto fixed = [&]() {
        li = b.state[kListIdx];
        if (!valid) return;
        nn = (int)PSC_IDX(b.nbr_n[li][i], kNB + 1, CHK_NBR);
        jn = b.nbr[li][i * kNB + sub];      // the lane's first neighbour (read without waiting for nn)
        ri = b.R[i];
        imi = (float)b.minv[2 * i];
        if (sub == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) { fi[a] = b.Ff[3 * i + a]; ti[a] = b.Tf[3 * i + a]; xr[a] = b.Xref[3 * i + a]; }
            im = b.minv[2 * i];
            iI = b.minv[2 * i + 1];
        }
    };
    if (early) {
        fixed();
        dep_wait();
    } else {
        dep_wait();
        fixed();
    }
    dep_launch();
    const int *const nbr = b.nbr[li];
    float *const hist = b.hist[li];
    // force and torque components a 2D disc has: F_x, F_y and T_z
    auto used = [](int q) { return DIM == 3 || q == 0 || q == 1 || q == 5; };
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double xi[3] = {0, 0, 0}, ui[3] = {0, 0, 0}, oi[3] = {0, 0, 0};
    int fail = 0;
    if (valid) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { xi[a] = b.X[3 * i + a]; ui[a] = b.U[3 * i + a]; oi[a] = b.Om[3 * i + a]; }
        const float4 pif = b.Xf[i];
        const float4 vi0 = b.Vf[2 * i], vi1 = b.Vf[2 * i + 1];
        const float uif[3] = {vi0.x, vi0.y, vi0.z};
        const float oif[3] = {vi0.w, vi1.x, vi1.y};
        for (int s = sub; s < nn; s += kLPP) {
            const int j = (int)PSC_IDX(jn, b.n, CHK_PART);
            if (s + kLPP < nn) jn = nbr[i * kNB + s + kLPP];
            float *hp = hist + ((size_t)i * kNB + s) * kH;
            // everything the pair may need, loaded at once (one round trip after j)
            const float4 pj = b.Xf[j];
            double xj[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int a = 0; a < 3; ++a) if (a < dim) xj[a] = b.X[3 * j + a];
            const double rj = b.R[j];
            const float4 vj0 = b.Vf[2 * j], vj1 = b.Vf[2 * j + 1];
            const float imj = (float)b.minv[2 * j];
            float4 *hp4 = reinterpret_cast<float4 *>(hp);
            const float4 h0 = hp4[0], h1 = hp4[1];
            // FP32 pre-filter on the position copies: pairs clearly apart skip the FP64 work
            float df[3] = {pj.x - pif.x, pj.y - pif.y, pj.z - pif.z};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a >= dim) { df[a] = 0.0f; continue; }
                if (g.periodic[a]) {
                    const float half = 0.5f * (float)g.n[a];
                    if (df[a] > half) df[a] -= (float)g.n[a];
                    else if (df[a] < -half) df[a] += (float)g.n[a];
                }
            }
            const bool was = h1.w != 0.0f;
            const float dpre = (pif.w + pj.w) - sqrtf(df[0] * df[0] + df[1] * df[1] + df[2] * df[2]);
            if (dpre < -b.reject) {
                // provably out of contact (the margin dwarfs the FP32 error)
                if (was) { hp4[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f); hp4[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f); }
                continue;
            }
            // separation X_j - X_i in FP64 (exact subtraction), minimum image; the periodic
            // shift is decided on the FP32 copy, exact for neighbours (|d| << n/2)
            double d[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (a >= dim) break;
                d[a] = __dsub_rn(xj[a], xi[a]);
                if (g.periodic[a]) {
                    const float half = 0.5f * (float)g.n[a], v = (float)d[a];
                    if (v > half) d[a] = __dsub_rn(d[a], (double)g.n[a]);
                    else if (v < -half) d[a] = __dadd_rn(d[a], (double)g.n[a]);
                }
            }
            // d^2 in FP64 with IEEE-rounded operations (bit-identical at both ends and in a
            // CPU reference); the contact decision of contact_sign (hostdev.cuh)
            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
            const double S = __dadd_rn(ri, rj);
            const ContactSign cs = contact_sign(d2, S);
            const bool ge0 = cs.ge0, gt0 = cs.gt0, exact = cs.exact;
            const float inv = cs.inv, dnf = cs.dnf;
            double dn = cs.dn;
            bool contact;
            if (!ph.adhesive) {
                contact = gt0;
            } else if (ge0) {
                contact = true;
            } else if (!was) {
                contact = false;
            } else {
                // a stretched neck persists while delta_N > -delta_C: decided in FP32 unless
                // the two agree to 1e-5, then with delta_N and delta_C in FP64
                const float Rf = pif.w * pj.w / (pif.w + pj.w);
                const float a0f = cbrtf((float)(9.0 * kPi) * ph.gamma * Rf * Rf / ph.Es);
                const float dCf = a0f * a0f * (float)ph.dc_coef / Rf;
                const float gap = dnf + dCf;
                if (fabsf(gap) > 1e-5f * dCf) {
                    contact = gap > 0.0f;
                } else {
                    if (!exact) dn = __dsub_rn(S, __dsqrt_rn(d2));
                    const double R64 = ri * rj / (ri + rj);
                    const double a064 = cbrt(9.0 * kPi * (double)ph.gamma * R64 * R64 / (double)ph.Es);
                    contact = dn > -(a064 * a064 * ph.dc_coef / R64);
                }
            }
            const float nv[3] = {(float)d[0] * inv, (float)d[1] * inv, (float)d[2] * inv};
            float hl[kH] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
            float fo[3], to[3];
            const float ujf[3] = {vj0.x, vj0.y, vj0.z};
            const float ojf[3] = {vj0.w, vj1.x, vj1.y};
            const float Rij = pif.w * pj.w / (pif.w + pj.w), msij = 1.0f / (imi + imj);
            if (contact_on_i(ph, dim, contact, nv, dnf, pif.w, pj.w, Rij, msij, uif, ujf, oif, ojf, hl, fo, to,
                             &fail)) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (used(a)) acc[a] += (double)fo[a];
                    if (used(3 + a)) acc[3 + a] += (double)to[a];
                }
            }
            if (was || hl[7] != 0.0f) {
                hp4[0] = make_float4(hl[0], hl[1], hl[2], hl[3]);
                hp4[1] = make_float4(hl[4], hl[5], hl[6], hl[7]);
            }
        }
    }
    // contacts with the walls of the non-periodic axes (the fluid's halfway bounce-back
    // planes at -1/2 and n - 1/2): lane `sub` takes axes sub, sub + kLPP, ...; the nearer wall
    // is a half-space of the same material at rest (R = r_i, m* = m_i). The overlap and the
    // decision are formed in FP64 with IEEE-rounded operations, as for the pairs.
#pragma unroll
    for (int a = 0; a < DIM; ++a) {       // unrolled: the per-axis arrays stay in registers
        if (!valid || a % kLPP != sub || g.periodic[a]) continue;
        const double lo_plane = 0.5 * (double)(g.n[a] - 1);
        const bool lower = xi[a] < lo_plane;
        const double dist = lower ? __dadd_rn(xi[a], 0.5) : __dsub_rn((double)g.n[a] - 0.5, xi[a]);
        const double dn = __dsub_rn(ri, dist);
        float4 *wp4 = reinterpret_cast<float4 *>(b.whist + ((size_t)i * 3 + a) * kH);
        if (dn < -2.0 * g.skin) {
            // far from this wall: no contact now, and none in the previous sub-step either
            // (the skin exceeds the largest pull-off separation and a call's displacement),
            // so the history is zero -- written, not read, to spare the round trip
            wp4[0] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            wp4[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            continue;
        }
        const float4 w0 = wp4[0], w1 = wp4[1];
        const bool was = w1.w != 0.0f;
        bool contact;
        if (!ph.adhesive) {
            contact = dn > 0.0;
        } else if (dn >= 0.0) {
            contact = true;
        } else if (!was) {
            contact = false;
        } else {
            const double a064 = cbrt(9.0 * kPi * (double)ph.gamma * ri * ri / (double)ph.Es);
            contact = dn > -(a064 * a064 * ph.dc_coef / ri);
        }
        if (contact || was) {
            float nv[3] = {0.0f, 0.0f, 0.0f};
            nv[a] = lower ? -1.0f : 1.0f;
            float hl[kH] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            float fo[3], to[3];
            const float zero[3] = {0.0f, 0.0f, 0.0f};
            const float4 vi0 = b.Vf[2 * i], vi1 = b.Vf[2 * i + 1];
            const float uif[3] = {vi0.x, vi0.y, vi0.z};
            const float oif[3] = {vi0.w, vi1.x, vi1.y};
            const float rif = (float)ri;
            const float msw = 1.0f / (float)b.minv[2 * i];
            if (contact_on_i(ph, dim, contact, nv, (float)dn, rif, 0.0f, rif, msw, uif, zero, oif, zero, hl, fo, to,
                             &fail)) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (used(c)) acc[c] += (double)fo[c];
                    if (used(3 + c)) acc[3 + c] += (double)to[c];
                }
            }
            wp4[0] = make_float4(hl[0], hl[1], hl[2], hl[3]);
            wp4[1] = make_float4(hl[4], hl[5], hl[6], hl[7]);
        }
    }
    // combine the kLPP partial sums (fixed butterfly order)
#pragma unroll
    for (int off = 1; off < kLPP; off <<= 1)
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (used(q)) acc[q] += __shfl_xor_sync(kFullMask, acc[q], off);
    if (fail) atomicAdd(&b.flags[1], 1);
    if (!valid || sub != 0) return;
    // Eq. 21, semi-implicit Euler, hydrodynamic force/torque frozen over the sub-steps
    double un[3], xn[3], on[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < dim) {
            un[a] = ui[a] + ph.dt * ((fi[a] + acc[a]) * im + ph.g[a]);
            xn[a] = xi[a] + ph.dt * un[a];
            // back into [0, n) on a periodic axis (a sub-step moves far less than a period)
            if (g.periodic[a]) {
                if (xn[a] < 0.0) xn[a] += (double)g.n[a];
                else if (xn[a] >= (double)g.n[a]) xn[a] -= (double)g.n[a];
            }
        } else {
            un[a] = ui[a];
            xn[a] = xi[a];
        }
        const bool spin = (dim == 3) || (a == 2);
        on[a] = spin ? oi[a] + ph.dt * (ti[a] + acc[3 + a]) * iI : oi[a];
    }
    const float disp2 = moved2(xn, xr, g.n, g.periodic, dim);
    if (disp2 > 0.25f * (float)(g.skin * g.skin)) atomicAdd(&b.flags[3], 1);
    // a quarter of the skin used: the next call rebuilds the list
    if (disp2 > 0.0625f * (float)(g.skin * g.skin)) b.state[kRebuildReq] = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) { b.Xo[3 * i + a] = xn[a]; b.Uo[3 * i + a] = un[a]; b.Omo[3 * i + a] = on[a]; }
    b.Xfo[i] = make_float4((float)xn[0], (float)xn[1], (float)xn[2], (float)ri);
    b.Vfo[2 * i] = make_float4((float)un[0], (float)un[1], (float)un[2], (float)on[0]);
    b.Vfo[2 * i + 1] = make_float4((float)on[1], (float)on[2], 0.0f, 0.0f);
}

}  // namespace

// ------------------------------------------------------------------------ host side
struct dem_ctx {
    dem_params p;
    lbm_ctx *fl;
    int n, cap_n;
    DemGeom g;
    DemPhys ph;
    double *X2, *U2, *Om2, *Xref, *minv;
    float4 *Xf[2];           // FP32 copies of the positions (current, next)
    float4 *Vf[2];           // FP32 copies of the velocities and spins (current, next)
    float reject;
    // CUDA graph of one dem_step call (even sub-step counts), keyed on what it captures
    cudaGraphExec_t gexec;
    const void *gkey[kDemKey];
    int gsub;
    int *bin_count, *bin_list;
    long long nbins;
    int *nbr_n[2], *nbr[2];
    float *hist[2];
    float *whist;            // [cap][3][kH] wall-contact history per particle and axis
    int **lists_dev;         // device copies of {nbr_n[0], nbr_n[1]}, {nbr[0], nbr[1]}, {hist[0], hist[1]}
    int *state;              // device words (kRebuildReq, kListIdx, kRebuildNow)
    int lists_valid;         // the device lists belong to the current particle set
    int force_rebuild;       // the host changed the particles: rebuild at the next call
    long long launches;
};

// Index of the current neighbour list (device word; synchronises the fluid's stream).
static int dem_list_index(dem_ctx *d, int *idx) {
    int h[kStateWords];
    cudaError_t e = cudaMemcpyAsync(h, d->state, sizeof(h), cudaMemcpyDeviceToHost, d->fl->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->fl->stream);
    *idx = h[kListIdx] & 1;
    return e == cudaSuccess;
}

lbm_ctx *dem_fluid(const dem_ctx *d) { return d ? d->fl : NULL; }

void dem_particles_changed(dem_ctx *d) {
    if (d) d->force_rebuild = 1;
}

int dem_upload_check(dem_ctx *d, int n, const double **ref, int **req, float *lim2) {
    if (!d || !d->lists_valid || d->force_rebuild || d->n != n || n <= 0 || !d->Xref || !d->state) return 0;
    *ref = d->Xref;
    *req = d->state + kRebuildReq;
    *lim2 = 0.0625f * (float)(d->g.skin * d->g.skin);   // the sub-step's own threshold
    return 1;
}

static void dfree(void **p) { if (*p) cudaFree(*p); *p = NULL; }

void dem_release(dem_ctx *d) {
    if (!d) return;
    dfree((void **)&d->X2); dfree((void **)&d->U2); dfree((void **)&d->Om2); dfree((void **)&d->Xref);
    dfree((void **)&d->minv);
    dfree((void **)&d->Xf[0]); dfree((void **)&d->Xf[1]);
    dfree((void **)&d->Vf[0]); dfree((void **)&d->Vf[1]);
    if (d->gexec) cudaGraphExecDestroy(d->gexec);
    dfree((void **)&d->lists_dev); dfree((void **)&d->state); dfree((void **)&d->whist);
    dfree((void **)&d->bin_count); dfree((void **)&d->bin_list);
    for (int k = 0; k < 2; ++k) { dfree((void **)&d->nbr_n[k]); dfree((void **)&d->nbr[k]); dfree((void **)&d->hist[k]); }
    free(d);
}

#define DCK(call, what)                                          \
    do {                                                         \
        lbm_status st_ = ctx_cuda(d->fl, (call), (what));        \
        if (st_ != LBM_OK) return st_;                           \
    } while (0)

// The DEM's state buffers are swapped with the fluid context's after every sub-step, so
// both sets must hold the fluid's full particle capacity (not just the current count).
static lbm_status dem_reserve(dem_ctx *d) {
    lbm_ctx *fl = d->fl;
    const int n = fl->np;
    const int cap = fl->np_cap;
    d->n = n;
    if (cap <= d->cap_n) return LBM_OK;
    dfree((void **)&d->X2); dfree((void **)&d->U2); dfree((void **)&d->Om2); dfree((void **)&d->Xref);
    dfree((void **)&d->minv);
    dfree((void **)&d->Xf[0]); dfree((void **)&d->Xf[1]);
    dfree((void **)&d->Vf[0]); dfree((void **)&d->Vf[1]);
    for (int k = 0; k < 2; ++k) { dfree((void **)&d->nbr_n[k]); dfree((void **)&d->nbr[k]); dfree((void **)&d->hist[k]); }
    const size_t v = (size_t)cap * 3 * sizeof(double);
    DCK(cudaMalloc(&d->Xf[0], (size_t)cap * sizeof(float4)), "cudaMalloc(DEM FP32 positions)");
    DCK(cudaMalloc(&d->Xf[1], (size_t)cap * sizeof(float4)), "cudaMalloc(DEM FP32 positions)");
    DCK(cudaMalloc(&d->Vf[0], (size_t)cap * 2 * sizeof(float4)), "cudaMalloc(DEM FP32 velocities)");
    DCK(cudaMalloc(&d->Vf[1], (size_t)cap * 2 * sizeof(float4)), "cudaMalloc(DEM FP32 velocities)");
    DCK(cudaMalloc(&d->minv, (size_t)cap * 2 * sizeof(double)), "cudaMalloc(DEM inverse mass)");
    DCK(cudaMalloc(&d->X2, v), "cudaMalloc(DEM X)");
    DCK(cudaMalloc(&d->U2, v), "cudaMalloc(DEM U)");
    DCK(cudaMalloc(&d->Om2, v), "cudaMalloc(DEM Omega)");
    DCK(cudaMalloc(&d->Xref, v), "cudaMalloc(DEM Xref)");
    dfree((void **)&d->whist);
    DCK(cudaMalloc(&d->whist, (size_t)cap * 3 * kH * sizeof(float)), "cudaMalloc(wall history)");
    DCK(cudaMemsetAsync(d->whist, 0, (size_t)cap * 3 * kH * sizeof(float), fl->stream), "memset");
    for (int k = 0; k < 2; ++k) {
        DCK(cudaMalloc(&d->nbr_n[k], (size_t)cap * sizeof(int)), "cudaMalloc(neighbour counts)");
        DCK(cudaMalloc(&d->nbr[k], (size_t)cap * kNB * sizeof(int)), "cudaMalloc(neighbour lists)");
        DCK(cudaMalloc(&d->hist[k], (size_t)cap * kNB * kH * sizeof(float)), "cudaMalloc(contact history)");
        DCK(cudaMemsetAsync(d->nbr_n[k], 0, (size_t)cap * sizeof(int), fl->stream), "memset");
        DCK(cudaMemsetAsync(d->hist[k], 0, (size_t)cap * kNB * kH * sizeof(float), fl->stream), "memset");
    }
    if (!d->state) {
        DCK(cudaMalloc(&d->state, kStateWords * sizeof(int)), "cudaMalloc(DEM state)");
        DCK(cudaMemsetAsync(d->state, 0, kStateWords * sizeof(int), fl->stream), "memset");
    }
    if (!d->lists_dev) DCK(cudaMalloc(&d->lists_dev, 6 * sizeof(int *)), "cudaMalloc(DEM list table)");
    int *tab[6] = {d->nbr_n[0], d->nbr_n[1], d->nbr[0], d->nbr[1], (int *)d->hist[0], (int *)d->hist[1]};
    DCK(cudaMemcpyAsync(d->lists_dev, tab, sizeof(tab), cudaMemcpyHostToDevice, fl->stream), "DEM list table");
    DCK(cudaStreamSynchronize(fl->stream), "sync");
    d->cap_n = cap;
    d->lists_valid = 0;
    return LBM_OK;
}

static lbm_status dem_setup_bins(dem_ctx *d) {
    lbm_ctx *fl = d->fl;
    const double side = 2.0 * fl->rmax + d->g.skin;
    long long nb = 1;
    for (int a = 0; a < 3; ++a) {
        d->g.nb[a] = (a < d->g.dim) ? (int)(fl->g.n[a] / side) : 1;
        if (d->g.nb[a] < 1) d->g.nb[a] = 1;
        d->g.bscale[a] = (double)d->g.nb[a] / fl->g.n[a];
        nb *= d->g.nb[a];
    }
    // bin capacity from the densest possible packing of the smallest admissible particles
    const double vol = (d->g.dim == 2) ? side * side : side * side * side;
    const double rmin = (d->g.dim == 2) ? 0.5 : 0.7071;
    const double pvol = (d->g.dim == 2) ? kPi * rmin * rmin : 4.0 / 3.0 * kPi * rmin * rmin * rmin;
    int cap = (int)(vol / pvol) + 8;
    if (cap > 256) cap = 256;
    if (nb != d->nbins || cap != d->g.bin_cap) {
        dfree((void **)&d->bin_count); dfree((void **)&d->bin_list);
        DCK(cudaMalloc(&d->bin_count, (size_t)nb * sizeof(int)), "cudaMalloc(DEM bins)");
        DCK(cudaMalloc(&d->bin_list, (size_t)nb * cap * sizeof(int)), "cudaMalloc(DEM bin lists)");
        d->nbins = nb;
        d->g.bin_cap = cap;
    }
    return LBM_OK;
}

extern "C" lbm_status dem_create(const dem_params *p, lbm_ctx *fluid, dem_ctx **out) {
    if (!fluid || !p || !out) return LBM_ERR_ARG;
    *out = NULL;
    if (!(p->E > 0) || !(p->poisson > -1.0 && p->poisson < 0.5) || !(p->density > 0) || !(p->dt_dem > 0) ||
        p->gamma < 0 || p->mu_f < 0 || p->theta_crit < 0 || p->alpha_n < 0 || p->k_t_scale < 0 ||
        p->eta_t_scale < 0 || (p->adhesive && !(p->gamma > 0))) {
        ctx_error(fluid, "invalid DEM parameters (E > 0, -1 < poisson < 1/2, density > 0, dt > 0, "
                         "non-negative friction/damping, gamma > 0 for JKR)");
        return LBM_ERR_ARG;
    }
    if (fluid->dem) { ctx_error(fluid, "the fluid context already has a DEM context"); return LBM_ERR_ARG; }
    dem_ctx *d = (dem_ctx *)calloc(1, sizeof(dem_ctx));
    if (!d) return LBM_ERR_OOM;
    d->p = *p;
    d->fl = fluid;
    d->g.dim = fluid->dim;
    for (int a = 0; a < 3; ++a) {
        d->g.n[a] = fluid->g.n[a];
        d->g.periodic[a] = fluid->g.periodic[a];
        d->g.inv_n[a] = 1.0 / fluid->g.n[a];
    }
    d->g.skin = p->skin > 0 ? p->skin : 0.5;
    d->ph.Es = (float)(p->E / (2.0 * (1.0 - p->poisson * p->poisson)));
    d->ph.Gs = (float)(p->E / (4.0 * (2.0 - p->poisson) * (1.0 + p->poisson)));
    d->ph.gamma = (float)p->gamma;
    d->ph.mu_f = (float)p->mu_f;
    d->ph.theta_crit = (float)p->theta_crit;
    d->ph.alpha_n = (float)p->alpha_n;
    d->ph.kt_scale = (float)p->k_t_scale;
    d->ph.etat_scale = (float)p->eta_t_scale;
    d->ph.dt = p->dt_dem;
    d->ph.density = p->density;
    for (int a = 0; a < 3; ++a) d->ph.g[a] = p->gravity[a];
    d->ph.adhesive = p->adhesive ? 1 : 0;
    d->ph.dc_coef = 1.0 / (2.0 * cbrt(6.0));
    fluid->dem = d;
    *out = d;
    return LBM_OK;
}

extern "C" lbm_status dem_destroy(dem_ctx *d) {
    if (!d) return LBM_OK;
    if (d->fl) { cudaStreamSynchronize(d->fl->stream); d->fl->dem = NULL; }
    dem_release(d);
    return LBM_OK;
}

// Launch with programmatic dependent launch (the kernel may start while its predecessor
// in the stream finishes; every DEM kernel begins with dep_wait()).
template <typename... KArgs, typename... Args>
static cudaError_t launch_dep(void (*kern)(KArgs...), unsigned blocks, unsigned threads, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Queue one dem_step call without touching host-side state, in two parts: the preparation
// (rebuild decision, FP32 copies, list rebuild when due), which reads only the particle
// state, and the sub-steps, which also read the fluid's F and T. The particle buffers
// alternate between the fluid context's and the DEM's own each sub-step (an odd count
// leaves them swapped; the caller swaps the pointers).
cudaError_t dem_enqueue_prep(dem_ctx *d, cudaStream_t s) {
    lbm_ctx *fl = d->fl;
    const int n = d->n;
    cudaError_t e = launch_dep(k_dem_decide, (unsigned)((d->nbins + 255) / 256 < 64 ? (d->nbins + 255) / 256 : 64),
                               256u, s, d->state, d->bin_count, d->nbins);
    if (e == cudaSuccess)
        e = launch_dep(k_dem_bin, (unsigned)((n + 127) / 128), 128u, s, d->g, n, (const double *)fl->dX,
                       (const double *)fl->dR, (const double *)fl->dU, (const double *)fl->dOm, d->Xf[0], d->Vf[0],
                       d->bin_count, d->bin_list, fl->flags, (const int *)d->state);
    if (e == cudaSuccess)
        e = launch_dep(k_dem_nbr, (unsigned)((n + 7) / 8), 256u, s, d->g, n, (const double *)fl->dX,
                       (const double *)fl->dR, (const float4 *)d->Xf[0], (const int *)d->bin_count,
                       (const int *)d->bin_list, (int *const *)d->lists_dev, (int *const *)(d->lists_dev + 2),
                       (float *const *)(d->lists_dev + 4), d->Xref, d->minv, d->ph.density, fl->flags,
                       (const int *)d->state);
    return e;
}

cudaError_t dem_enqueue_substeps(dem_ctx *d, int substeps, cudaStream_t s) {
    lbm_ctx *fl = d->fl;
    const int n = d->n;
    cudaError_t e = cudaSuccess;
    DemBufs b;
    b.n = n;
    b.R = fl->dR;
    b.Ff = fl->dF;
    b.Tf = fl->dT;
    b.Xref = d->Xref;
    for (int k = 0; k < 2; ++k) { b.nbr_n[k] = d->nbr_n[k]; b.nbr[k] = d->nbr[k]; b.hist[k] = d->hist[k]; }
    b.state = d->state;
    b.whist = d->whist;
    b.minv = d->minv;
    b.flags = fl->flags;
    b.reject = d->reject;
    const int threads = 128;
    const int blocks = (int)(((long long)n * kLPP + threads - 1) / threads);
    double *X[2] = {fl->dX, d->X2}, *U[2] = {fl->dU, d->U2}, *Om[2] = {fl->dOm, d->Om2};
    for (int k = 0; k < substeps && e == cudaSuccess; ++k) {
        const int src = k & 1, dst = src ^ 1;
        b.X = X[src]; b.U = U[src]; b.Om = Om[src]; b.Xf = d->Xf[src]; b.Vf = d->Vf[src];
        b.Xo = X[dst]; b.Uo = U[dst]; b.Omo = Om[dst]; b.Xfo = d->Xf[dst]; b.Vfo = d->Vf[dst];
        const int early = k > 0 ? 1 : 0;
        if (d->g.dim == 2) e = launch_dep(k_dem_substep<2>, (unsigned)blocks, (unsigned)threads, s, d->g, d->ph, b, early);
        else e = launch_dep(k_dem_substep<3>, (unsigned)blocks, (unsigned)threads, s, d->g, d->ph, b, early);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

static cudaError_t dem_enqueue(dem_ctx *d, int substeps) {
    cudaError_t e = dem_enqueue_prep(d, d->fl->stream);
    if (e == cudaSuccess) e = dem_enqueue_substeps(d, substeps, d->fl->stream);
    return e;
}

// The host side of a call before its kernels: buffers, bins, the list's state (memsets on
// the stream when the list starts again or a rebuild is forced) and the rejection margin.
// *run = 0 when the call has nothing to do.
lbm_status dem_prepare(dem_ctx *d, int substeps, int *run) {
    lbm_ctx *fl = d->fl;
    *run = 0;
    if (substeps < 0) { ctx_error(fl, "substeps must be >= 0"); return LBM_ERR_ARG; }
    if (fl->np == 0 || substeps == 0) return LBM_OK;
    if (fl->np != d->n) d->lists_valid = 0;
    lbm_status st = dem_reserve(d);
    if (st != LBM_OK) return st;
    st = dem_setup_bins(d);
    if (st != LBM_OK) return st;
    if (!d->lists_valid) {
        // no list to carry contact history over from (first call, a new particle count, or
        // a checkpoint without a DEM section): every pair starts without history
        for (int k = 0; k < 2; ++k)
            DCK(cudaMemsetAsync(d->nbr_n[k], 0, (size_t)d->n * sizeof(int), fl->stream), "memset");
        DCK(cudaMemsetAsync(d->whist, 0, (size_t)d->n * 3 * kH * sizeof(float), fl->stream), "memset");
        d->force_rebuild = 1;
    }
    if (d->force_rebuild) {
        // any nonzero request word rebuilds the list at the start of this call
        DCK(cudaMemsetAsync(d->state + kRebuildReq, 0xff, sizeof(int), fl->stream), "memset");
        d->force_rebuild = 0;
    }
    // largest delta_C of any pair (R <= r_max / 2) plus a margin far above the FP32 error of
    // the position copies
    int nmax = 1;
    for (int a = 0; a < d->g.dim; ++a) nmax = fl->g.n[a] > nmax ? fl->g.n[a] : nmax;
    d->g.margin = (float)(1e-3 + 8.0 * nmax / 16777216.0);
    const double Es = d->p.E / (2.0 * (1.0 - d->p.poisson * d->p.poisson));
    const double Rm = 0.5 * fl->rmax;
    const double a0 = cbrt(9.0 * kPi * d->p.gamma * Rm * Rm / Es);
    const double dC = d->p.adhesive ? a0 * a0 / (2.0 * cbrt(6.0) * Rm) : 0.0;
    d->reject = (float)(dC + d->g.margin);
    if (dC >= d->g.skin) {
        ctx_error(fl, "the neighbour-list skin %g must exceed the largest JKR pull-off separation %g "
                      "(dem_params.skin)", d->g.skin, dC);
        return LBM_ERR_ARG;
    }
    *run = 1;
    return LBM_OK;
}

// Everything a call's kernels capture (a CUDA graph of the call is valid while this is unchanged).
void dem_graph_key(const dem_ctx *d, const void *key[kDemKey]) {
    const lbm_ctx *fl = d->fl;
    unsigned rbits;
    memcpy(&rbits, &d->reject, sizeof(rbits));
    const void *k[kDemKey] = {d->Vf[0], fl->dX, fl->dU, fl->dOm, fl->dR, fl->dF, fl->dT, d->X2, d->U2, d->Om2,
                              d->Xf[0], d->minv, d->bin_count, (const void *)(size_t)d->n, (const void *)(size_t)rbits,
                              (const void *)(size_t)(d->g.nb[0] + 4096LL * (d->g.nb[1] + 4096LL * d->g.nb[2])),
                              (const void *)(size_t)d->g.bin_cap};
    for (int i = 0; i < kDemKey; ++i) key[i] = k[i];
}

// The host bookkeeping after a call's kernels were queued (an even sub-step count leaves
// every buffer where it started; an odd one, queued directly, swaps them).
void dem_after_call(dem_ctx *d, int substeps, int swap) {
    lbm_ctx *fl = d->fl;
    if (swap && (substeps & 1)) {
        double *t;
        t = fl->dX; fl->dX = d->X2; d->X2 = t;
        t = fl->dU; fl->dU = d->U2; d->U2 = t;
        t = fl->dOm; fl->dOm = d->Om2; d->Om2 = t;
    }
    const int kernels = 3 + substeps;
    d->lists_valid = 1;
    d->launches += kernels;
    fl->launches += kernels;
    fl->bins_valid = 0;   // particles moved: the fluid re-bins before its next step
}

extern "C" lbm_status dem_step(dem_ctx *d, int substeps) {
    NvtxRange nvtx_("dem_step");
    if (!d) return LBM_ERR_ARG;
    lbm_ctx *fl = d->fl;
    int run = 0;
    lbm_status st = dem_prepare(d, substeps, &run);
    if (st != LBM_OK || !run) return st;
    // even sub-step counts leave every buffer where it started, so the whole call can be
    // replayed from one CUDA graph, keyed on every pointer and size it was captured with
    // (the list buffers in use are chosen on the device)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    DCK(cudaStreamIsCapturing(fl->stream, &cs), "cudaStreamIsCapturing");
    const void *key[kDemKey];
    dem_graph_key(d, key);
    if (substeps % 2 == 0 && cs == cudaStreamCaptureStatusNone) {
        bool same = d->gexec && d->gsub == substeps;
        for (int k = 0; same && k < kDemKey; ++k) same = (d->gkey[k] == key[k]);
        if (!same) {
            if (d->gexec) { cudaGraphExecDestroy(d->gexec); d->gexec = NULL; }
            cudaGraph_t graph = NULL;
            DCK(cudaStreamBeginCapture(fl->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
            cudaError_t eq = dem_enqueue(d, substeps);
            cudaError_t ec = cudaStreamEndCapture(fl->stream, &graph);
            DCK(eq, "DEM kernels (capture)");
            DCK(ec, "cudaStreamEndCapture");
            cudaError_t ei = cudaGraphInstantiate(&d->gexec, graph, 0);
            cudaGraphDestroy(graph);
            DCK(ei, "cudaGraphInstantiate");
            d->gsub = substeps;
            for (int k = 0; k < kDemKey; ++k) d->gkey[k] = key[k];
        }
        DCK(cudaGraphLaunch(d->gexec, fl->stream), "cudaGraphLaunch");
        dem_after_call(d, substeps, 0);
        return LBM_OK;
    }
    DCK(dem_enqueue(d, substeps), "DEM kernels");
    dem_after_call(d, substeps, 1);
    return LBM_OK;
}

// ---------------------------------------------------------------- checkpoint section
// Layout: {magic, n, kNB, kH} as int64, then the current list: counts (n int32), slots
// (n x kNB int32), history (n x kNB x kH float), then the wall-contact history (n x 3 x kH
// float). The next dem_step rebuilds the list from the positions and carries the history
// over from this one, so a run resumed from it continues as the saved run did.
static const long long kDemMagic = 0x50534344454d3032LL;   // "PSCDEM02"

size_t dem_state_bytes(const dem_ctx *d) {
    if (!d || !d->lists_valid || d->n <= 0) return 0;
    const size_t n = (size_t)d->n;
    return 4 * sizeof(long long) + n * sizeof(int) + n * kNB * sizeof(int) + n * kNB * kH * sizeof(float) +
           n * 3 * kH * sizeof(float);
}

lbm_status dem_state_save(dem_ctx *d, char *dst) {
    if (dem_state_bytes(d) == 0) return LBM_OK;
    const size_t n = (size_t)d->n;
    const long long h[4] = {kDemMagic, d->n, kNB, kH};
    memcpy(dst, h, sizeof(h));
    dst += sizeof(h);
    cudaStream_t s = d->fl->stream;
    int cur = 0;
    if (!dem_list_index(d, &cur)) return ctx_cuda(d->fl, cudaGetLastError(), "read DEM state");
    DCK(cudaMemcpyAsync(dst, d->nbr_n[cur], n * sizeof(int), cudaMemcpyDeviceToHost, s), "save DEM counts");
    dst += n * sizeof(int);
    DCK(cudaMemcpyAsync(dst, d->nbr[cur], n * kNB * sizeof(int), cudaMemcpyDeviceToHost, s), "save DEM lists");
    dst += n * kNB * sizeof(int);
    DCK(cudaMemcpyAsync(dst, d->hist[cur], n * kNB * kH * sizeof(float), cudaMemcpyDeviceToHost, s),
        "save DEM history");
    dst += n * kNB * kH * sizeof(float);
    DCK(cudaMemcpyAsync(dst, d->whist, n * 3 * kH * sizeof(float), cudaMemcpyDeviceToHost, s), "save wall history");
    return LBM_OK;
}

void dem_state_clear(dem_ctx *d) {
    if (d) d->lists_valid = 0;
}

lbm_status dem_state_load(dem_ctx *d, const char *src, size_t size) {
    long long h[4];
    if (size < sizeof(h)) { ctx_error(d->fl, "DEM checkpoint section truncated"); return LBM_ERR_ARG; }
    memcpy(h, src, sizeof(h));
    if (h[0] != kDemMagic || h[1] != d->fl->np || h[2] != kNB || h[3] != kH) {
        ctx_error(d->fl, "DEM checkpoint section does not match this context");
        return LBM_ERR_ARG;
    }
    const size_t n = (size_t)h[1];
    if (size < sizeof(h) + n * sizeof(int) + n * kNB * sizeof(int) + n * kNB * kH * sizeof(float) +
                   n * 3 * kH * sizeof(float)) {
        ctx_error(d->fl, "DEM checkpoint section truncated");
        return LBM_ERR_ARG;
    }
    lbm_status st = dem_reserve(d);
    if (st != LBM_OK) return st;
    src += sizeof(h);
    cudaStream_t s = d->fl->stream;
    int cur = 0;
    if (!dem_list_index(d, &cur)) return ctx_cuda(d->fl, cudaGetLastError(), "read DEM state");
    DCK(cudaMemcpyAsync(d->nbr_n[cur], src, n * sizeof(int), cudaMemcpyHostToDevice, s), "load DEM counts");
    src += n * sizeof(int);
    DCK(cudaMemcpyAsync(d->nbr[cur], src, n * kNB * sizeof(int), cudaMemcpyHostToDevice, s), "load DEM lists");
    src += n * kNB * sizeof(int);
    DCK(cudaMemcpyAsync(d->hist[cur], src, n * kNB * kH * sizeof(float), cudaMemcpyHostToDevice, s),
        "load DEM history");
    src += n * kNB * kH * sizeof(float);
    DCK(cudaMemcpyAsync(d->whist, src, n * 3 * kH * sizeof(float), cudaMemcpyHostToDevice, s), "load wall history");
    DCK(cudaStreamSynchronize(s), "sync");
    d->n = (int)n;
    d->lists_valid = 1;
    d->force_rebuild = 1;    // the restored list is carried over into a list of the restored positions
    return LBM_OK;
}

extern "C" lbm_status dem_get_particles(dem_ctx *d, double *X, double *U, double *Om, int on_device) {
    if (!d) return LBM_ERR_ARG;
    lbm_ctx *fl = d->fl;
    const size_t v = (size_t)fl->np * 3 * sizeof(double);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (fl->np == 0) return LBM_OK;
    if (X) DCK(cudaMemcpyAsync(X, fl->dX, v, k, fl->stream), "copy X");
    if (U) DCK(cudaMemcpyAsync(U, fl->dU, v, k, fl->stream), "copy U");
    if (Om) DCK(cudaMemcpyAsync(Om, fl->dOm, v, k, fl->stream), "copy Omega");
    if (!on_device) return ctx_check_flags(fl);
    return LBM_OK;
}

// Contacts as canonical pairs i < j (sorted) and the history seen from i.
extern "C" lbm_status dem_get_contacts(dem_ctx *d, int *pairs, double *hist, int cap, int *nout) {
    if (!d || !nout) return LBM_ERR_ARG;
    lbm_ctx *fl = d->fl;
    *nout = 0;
    if (!d->lists_valid || d->n == 0) return ctx_check_flags(fl);
    const int n = d->n;
    int cur = 0;
    if (!dem_list_index(d, &cur)) return ctx_cuda(fl, cudaGetLastError(), "read DEM state");
    int *hn = (int *)malloc((size_t)n * sizeof(int));
    int *hb = (int *)malloc((size_t)n * kNB * sizeof(int));
    float *hh = (float *)malloc((size_t)n * kNB * kH * sizeof(float));
    if (!hn || !hb || !hh) { free(hn); free(hb); free(hh); return LBM_ERR_OOM; }
    cudaError_t e = cudaMemcpyAsync(hn, d->nbr_n[cur], (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, fl->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb, d->nbr[cur], (size_t)n * kNB * sizeof(int), cudaMemcpyDeviceToHost, fl->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hh, d->hist[cur], (size_t)n * kNB * kH * sizeof(float), cudaMemcpyDeviceToHost, fl->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(fl->stream);
    if (e != cudaSuccess) { free(hn); free(hb); free(hh); return ctx_cuda(fl, e, "copy contacts"); }
    int k = 0;
    lbm_status st = LBM_OK;
    for (int i = 0; i < n; ++i) {
        for (int s = 0; s < hn[i]; ++s) {
            const int j = hb[i * kNB + s];
            const float *h = hh + ((size_t)i * kNB + s) * kH;
            if (j <= i || h[7] == 0.0f) continue;
            if (k < cap) {
                if (pairs) { pairs[2 * k] = i; pairs[2 * k + 1] = j; }
                if (hist) for (int q = 0; q < 7; ++q) hist[7 * (size_t)k + q] = (double)h[q];
            } else {
                st = LBM_ERR_OVERFLOW;
            }
            ++k;
        }
    }
    free(hn); free(hb); free(hh);
    *nout = k;
    if (st != LBM_OK) { ctx_error(fl, "contact buffer holds %d pairs, %d needed", cap, k); return st; }
    return ctx_check_flags(fl);
}

// Wall contacts of the last sub-step as (particle, axis) pairs sorted by particle, with the
// history of each (7 doubles: sliding spring xyz, twist, rolling spring xyz).
extern "C" lbm_status dem_get_wall_contacts(dem_ctx *d, int *pw, double *hist, int cap, int *nout) {
    if (!d || !nout) return LBM_ERR_ARG;
    lbm_ctx *fl = d->fl;
    *nout = 0;
    if (!d->lists_valid || d->n == 0 || !d->whist) return ctx_check_flags(fl);
    const size_t cnt = (size_t)d->n * 3 * kH;
    float *hw = (float *)malloc(cnt * sizeof(float));
    if (!hw) return LBM_ERR_OOM;
    cudaError_t e = cudaMemcpyAsync(hw, d->whist, cnt * sizeof(float), cudaMemcpyDeviceToHost, fl->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(fl->stream);
    if (e != cudaSuccess) { free(hw); return ctx_cuda(fl, e, "copy wall history"); }
    int k = 0;
    lbm_status st = LBM_OK;
    for (int i = 0; i < d->n; ++i)
        for (int a = 0; a < 3; ++a) {
            const float *h = hw + ((size_t)i * 3 + a) * kH;
            if (h[7] == 0.0f) continue;
            if (k < cap) {
                if (pw) { pw[2 * k] = i; pw[2 * k + 1] = a; }
                if (hist) for (int q = 0; q < 7; ++q) hist[7 * (size_t)k + q] = (double)h[q];
            } else {
                st = LBM_ERR_OVERFLOW;
            }
            ++k;
        }
    free(hw);
    *nout = k;
    if (st != LBM_OK) { ctx_error(fl, "wall contact buffer holds %d entries, %d needed", cap, k); return st; }
    return ctx_check_flags(fl);
}

extern "C" lbm_status dem_get_info(dem_ctx *d, long long *out, int n) {
    if (!d || !out || n < 1) return LBM_ERR_ARG;
    lbm_ctx *fl = d->fl;
    int h[4] = {0, 0, 0, 0}, st[kStateWords] = {0, 0, 0, 0};
    DCK(cudaMemcpyAsync(h, fl->flags, sizeof(h), cudaMemcpyDeviceToHost, fl->stream), "read flags");
    if (d->state) DCK(cudaMemcpyAsync(st, d->state, sizeof(st), cudaMemcpyDeviceToHost, fl->stream), "read state");
    DCK(cudaStreamSynchronize(fl->stream), "sync");
    long long vals[6] = {d->launches, h[1], h[2], h[3], d->n, st[kRebuilds]};
    for (int i = 0; i < n && i < 6; ++i) out[i] = vals[i];
    return LBM_OK;
}

// the bounds-check word of this translation unit (see psc_internal.h)
PSC_CHECK_READER(psc_chk_take_dem)
