// psc_pair.cuh -- the particle-tile path of the PSC collide-stream step with two cells per
// thread (included by psc_kernels.cuh inside namespace psc, after the shared helpers).
//
// A 128-thread block owns one tile (32 x 8 cells in 2D, 32 x 4 x 2 in 3D). Each warp takes
// two rows of it (2D: rows 2w and 2w + 1; 3D: row w at both z), each lane the two cells of
// its column, so every per-candidate step -- the record loads, the row test, the loop
// control, the force reduction -- is paid once per two cells. The per-cell arithmetic runs
// on pairs (cell a, cell b); in FP32 a pair is one packed register pair and one FFMA2 /
// FADD2 / FMUL2 instruction does both cells.
//
// Per tile, in the order of the paper's steps: records of the tile's candidates to shared
// memory; pull (Eq. 1, 6) and moments (Eq. 5); the candidates that can reach either row;
// one pass over them for the solid fraction (Table 1, Eq. 15-18), the u_s moments of the
// collision and each candidate's momentum-exchange bracket; weights (Eq. 9, 13); collision
// (Eq. 2-4, 10, 12) and store; force and torque (Eq. 14) per candidate, summed over the warp
// and, after the next tile's barrier, over the block.

constexpr int kPThreads = 128;
constexpr int kPWarps = kPThreads / 32;

// Pairs of the compute type: FP32 on the packed sm_100 instructions, FP64 as two scalars.
template <typename T> struct Pr;
template <> struct Pr<float> {
    using V = float2;
    static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ V sp(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ V add(V x, V y) { return __fadd2_rn(x, y); }
    static __device__ __forceinline__ V sub(V x, V y) { return __fadd2_rn(x, make_float2(-y.x, -y.y)); }
    static __device__ __forceinline__ V mul(V x, V y) { return __fmul2_rn(x, y); }
    static __device__ __forceinline__ V fma(V x, V y, V z) { return __ffma2_rn(x, y, z); }
};
template <> struct Pr<double> {
    using V = double2;
    static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ V sp(double a) { return make_double2(a, a); }
    static __device__ __forceinline__ V add(V x, V y) { return make_double2(x.x + y.x, x.y + y.y); }
    static __device__ __forceinline__ V sub(V x, V y) { return make_double2(x.x - y.x, x.y - y.y); }
    static __device__ __forceinline__ V mul(V x, V y) { return make_double2(x.x * y.x, x.y * y.y); }
    static __device__ __forceinline__ V fma(V x, V y, V z) {
        return make_double2(::fma(x.x, y.x, z.x), ::fma(x.y, y.y, z.y));
    }
};

// e_i . v on pairs (additions only, as edot)
template <class L, typename T>
__device__ __forceinline__ typename Pr<T>::V edot2(const int i, const typename Pr<T>::V vx,
                                                   const typename Pr<T>::V vy, const typename Pr<T>::V vz) {
    using P = Pr<T>;
    const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
    typename P::V r = P::sp((T)0);
    bool first = true;
    auto acc = [&](int e, typename P::V v) {
        if (!e) return;
        if (first) { r = e > 0 ? v : P::sub(P::sp((T)0), v); first = false; }
        else r = e > 0 ? P::add(r, v) : P::sub(r, v);
    };
    acc(ex, vx);
    acc(ey, vy);
    acc(ez, vz);
    return r;
}

// eps_n = min(1, sum eps), B_n by Eq. 9 at eps_n and the normalisation c_B of Eq. 13
// (B_{n,s} = c_B eps_s); original scheme: B_n = sum_s B(eps_s) (Eq. 8), c_B = 1.
template <int PSC, typename T>
__device__ __forceinline__ void psc_weights(const T seps, const T tmh, T &Bn, T &cB) {
    Bn = (T)0;
    cB = (T)0;
    if (seps > (T)0) {
        if (PSC == 0) {
            if (seps < (T)1) {
                cB = tmh / (((T)1 - seps) + tmh);
                Bn = seps * cB;
            } else {
                Bn = (T)1;
                cB = (T)1 / seps;
            }
        } else {
            Bn = seps;
            cB = (T)1;
        }
    }
}

// Tile totals of the per-warp partial forces (fixed warp order), one FP64 atomic per particle
// and component; the particle indices come from the records in global memory (the shared
// copy may already hold the next tile's).
template <class L, typename T>
__device__ __forceinline__ void pair_flush(const int cnt, const T *recs, const T *part, const unsigned *mask,
                                           const Parts &pd, const int tid) {
    constexpr int NC = (L::D == 2) ? 3 : 6;
    for (int idx = tid; idx < cnt * NC; idx += kPThreads) {
        const int k = idx / NC, q = idx - k * NC;
        T sum = 0;
        bool any = false;
#pragma unroll
        for (int w = 0; w < kPWarps; ++w) {
            if ((mask[w] >> k) & 1u) { sum += part[(w * kPairCap + k) * NC + q]; any = true; }
        }
        if (any && sum != (T)0) {
            const int pid = (int)PSC_IDX(bits_id(recs[k * RW + R_ID]), pd.n, CHK_PART);
            double *dst;
            if (L::D == 2) dst = (q < 2) ? &pd.F[3 * pid + q] : &pd.T[3 * pid + 2];
            else dst = (q < 3) ? &pd.F[3 * pid + q] : &pd.T[3 * pid + q - 3];
            atomicAdd(dst, -(double)sum);
        }
    }
}

// The lane's two cells, tile-relative: one column (the lane), both of the warp's rows.
template <class L>
struct PairCells {
    int xA, xB, yA, yB, zA, zB;
    __device__ __forceinline__ PairCells(const int lane, const int warp) {
        xA = xB = lane;
        yA = (L::D == 2) ? 2 * warp : warp;
        yB = (L::D == 2) ? 2 * warp + 1 : warp;
        zA = 0;
        zB = (L::D == 2) ? 0 : 1;
    }
};

// Pull of the lane's two cells (raw values for 16-bit storage, which folds its scale).
template <class L, typename S>
__device__ __forceinline__ void pull_pair(const S *__restrict__ fin, const Geom &g, const PhysT<typename Store<S>::T> &ph,
                                          const bool interior, const int xA, const int xB, const int yA,
                                          const int yB, const int zA, const int zB, const long long cellA,
                                          const long long cellB, const bool actA, const bool actB,
                                          typename Store<S>::T *da, typename Store<S>::T *db) {
    constexpr bool SC = Store<S>::kScaled;
    if (interior) {     // both cells with the same fixed offsets (one copy of the load code)
        const long long N = g.ncell, sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
        const S *ba = fin + cellA, *bb = fin + cellB;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            const long long o = (long long)i * N - (L::ex(i) + L::ey(i) * sy + L::ez(i) * sz);
            const long long oa = PSC_OFF(cellA, o, L::Q * N, CHK_POP), ob = PSC_OFF(cellB, o, L::Q * N, CHK_POP);
            da[i] = SC ? Store<S>::ldr(ba, oa) : Store<S>::ld(ba, oa, ph.sc);
            db[i] = SC ? Store<S>::ldr(bb, ob) : Store<S>::ld(bb, ob, ph.sc);
        }
        return;
    }
    pull_q<L, S, SC>(fin, g, xA, yA, zA, cellA, false, actA, ph.sc, da);
    pull_q<L, S, SC>(fin, g, xB, yB, zB, cellB, false, actB, ph.sc, db);
}

// Store of velocity i at the lane's two cells (values already scaled for 16-bit storage).
template <typename S>
__device__ __forceinline__ void store_pair(S *__restrict__ fout, const long long iA, const long long iB,
                                           const typename Store<S>::T a, const typename Store<S>::T b,
                                           const bool actA, const bool actB, const long long lim) {
    (void)lim;   // the extent the bounds-checked build tests the indices of active cells against
    if (actA) Store<S>::str(fout, PSC_IDX(iA, lim, CHK_POP), a);
    if (actB) Store<S>::str(fout, PSC_IDX(iB, lim, CHK_POP), b);
}

template <class L> constexpr int pair_nslot() { return 4; }

template <class L, typename T> __host__ __device__ constexpr size_t pair_smem_bytes() {
    // records [2][kPairCap][RW] | partials [2][kPWarps][kPairCap][NC] | brackets
    // [kPWarps][NSLOT + 1][NC][32] pairs (the last slot is scratch for further candidates)
    return (size_t)2 * kPairCap * RW * sizeof(T) + (size_t)2 * kPWarps * kPairCap * ((L::D == 2) ? 3 : 6) * sizeof(T) +
           (size_t)kPWarps * (pair_nslot<L>() + 1) * ((L::D == 2) ? 3 : 6) * 32 * 2 * sizeof(T);
}

template <class L, typename S, int PSC>
__device__ __forceinline__ void psc_tile_pair(const uint2 ent, const int cnt, const S *__restrict__ fin,
                                              S *__restrict__ fout, const Geom &g,
                                              const PhysT<typename Store<S>::T> &ph, const Tiles &tl,
                                              const Parts &pd, int *flags, typename Store<S>::T *srec,
                                              typename Store<S>::T *part, unsigned *s_mask, const int prev_cnt,
                                              const typename Store<S>::T *prev_recs,
                                              const typename Store<S>::T *prev_part, const unsigned *prev_mask,
                                              typename Pr<typename Store<S>::T>::V *sbr) {
    using T = typename Store<S>::T;
    using P = Pr<T>;
    using V = typename P::V;
    constexpr int Q = L::Q;
    constexpr int NC = (L::D == 2) ? 3 : 6;
    constexpr int NSLOT = pair_nslot<L>();
    const int cap = tl.cap;

    const unsigned tile = (unsigned)PSC_IDX(ent.x, (long long)g.nt[0] * g.nt[1] * g.nt[2], CHK_TILE);
    const unsigned ty = ent.y & 0xffffu, tz = ent.y >> 16;
    const int x0 = (int)(tile - (unsigned)g.nt[0] * (ty + (unsigned)g.nt[1] * tz)) * L::TX;
    const int y0 = (int)ty * L::TY;
    const int z0 = (int)tz * L::TZ;
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int tid = lane + 32 * warp;
    // the warp's two rows, tile-relative (the candidate row test covers both)
    const int ryA = (L::D == 2) ? 2 * warp : warp, ryB = (L::D == 2) ? 2 * warp + 1 : warp;
    const int rzA = 0, rzB = (L::D == 2) ? 0 : 1;
    const PairCells<L> pc(lane, warp);
    const int xA = x0 + pc.xA, xB = x0 + pc.xB;
    const int yA = y0 + pc.yA, yB = y0 + pc.yB, zA = z0 + pc.zA, zB = z0 + pc.zB;
    const bool actA = cell_active<L>(g, xA, yA, zA);
    const bool actB = cell_active<L>(g, xB, yB, zB);
    const long long cellA = xA + (long long)g.n[0] * (yA + (long long)g.n[1] * zA);
    const long long cellB = xB + (long long)g.n[0] * (yB + (long long)g.n[1] * zB);
    const long long N = g.ncell;
    const T *recs = reinterpret_cast<const T *>(tl.blocks) + (size_t)tile * block_elems<T>(cap) + head_elems<T>();

    // ---- records: this thread's share, loaded before the pull, stored after it
    constexpr int kRecWords = (kPairCap * RW + kPThreads - 1) / kPThreads;
    T rw[kRecWords];
    const int nwords = cnt * RW;
#pragma unroll
    for (int j = 0; j < kRecWords; ++j) {
        const int w = tid + j * kPThreads;
        rw[j] = (w < nwords) ? recs[w] : (T)0;
    }

    // ---- pull and moments (Eq. 1, 5, 6)
    const bool interior = x0 >= 1 && x0 + L::TX < g.n[0] && y0 >= 1 && y0 + L::TY < g.n[1] &&
                          (L::D == 2 || (z0 >= 1 && z0 + L::TZ < g.n[2]));
    // 16-bit storage: the stored values carry the scale s; they are summed as stored and the
    // sums unscaled once, and the outputs are formed scaled (s folded into the weights)
    constexpr bool SC = Store<S>::kScaled;
    T da[Q], db[Q];
    pull_pair<L, S>(fin, g, ph, interior, xA, xB, yA, yB, zA, zB, cellA, cellB, actA, actB, da, db);
    V df[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = P::mk(da[i], db[i]);
    V drho = df[0], jx = P::sp((T)0), jy = P::sp((T)0), jz = P::sp((T)0);
#pragma unroll
    for (int i = 1; i < Q; ++i) drho = P::add(drho, df[i]);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (L::ex(i)) jx = L::ex(i) > 0 ? P::add(jx, df[i]) : P::sub(jx, df[i]);
        if (L::ey(i)) jy = L::ey(i) > 0 ? P::add(jy, df[i]) : P::sub(jy, df[i]);
        if (L::ez(i)) jz = L::ez(i) > 0 ? P::add(jz, df[i]) : P::sub(jz, df[i]);
    }
    const T ssc = SC ? (T)ph.sc.x : (T)1;           // s (the stored values are s d)
    if (SC) {
        const V is = P::sp((T)ph.sc.y);
        drho = P::mul(drho, is); jx = P::mul(jx, is); jy = P::mul(jy, is); jz = P::mul(jz, is);
    }
    const V rho = P::add(P::sp((T)1), drho);
    const V irho = P::mk((T)1 / rho.x, (T)1 / rho.y);
    const V hF0 = P::sp((T)0.5 * ph.F[0]), hF1 = P::sp((T)0.5 * ph.F[1]), hF2 = P::sp((T)0.5 * ph.F[2]);
    const V ux = P::mul(P::add(jx, hF0), irho);
    const V uy = P::mul(P::add(jy, hF1), irho);
    const V uz = P::mul(P::add(jz, hF2), irho);
    if ((actA && !(rho.x > (T)0)) || (actB && !(rho.y > (T)0))) atomicOr(flags, 1);
    // p = F/2 - j: the fluid part of the per-cell momentum exchange (Eq. 14)
    const V px = P::sub(hF0, jx), py = P::sub(hF1, jy), pz = P::sub(hF2, jz);

#pragma unroll
    for (int j = 0; j < kRecWords; ++j) {
        const int w = tid + j * kPThreads;
        if (w < nwords) srec[w] = rw[j];
    }
    // the block's one barrier per tile: records staged, and every warp is done with the
    // previous tile, whose partial forces are added up now
    __syncthreads();
    pair_flush<L, T>(prev_cnt, prev_recs, prev_part, prev_mask, pd, tid);

    // ---- candidates that can reach either row (one lane per candidate, ballot)
    const T cxA = (T)pc.xA, cxB = (T)pc.xB;
    const T cyA = (T)pc.yA, cyB = (T)pc.yB, czA = (T)pc.zA, czB = (T)pc.zB;
    const T xmax = (T)(min(L::TX, g.n[0] - x0) - 1);
    unsigned wmask;
    {
        bool rel = false;
        if (lane < cnt) {
            const Vec4<T> a = ld4<T>(srec + lane * RW);
            rel = row_hits<L, T>(g, a.x, a.y, a.z, a.w + ph.h, (T)ryA, (T)rzA, xmax) ||
                  row_hits<L, T>(g, a.x, a.y, a.z, a.w + ph.h, (T)ryB, (T)rzB, xmax);
        }
        wmask = __ballot_sync(kFull, rel);
    }

    // ---- one pass over the candidates: eps_s, u_s moments, brackets
    V seps = P::sp((T)0), mx = seps, my = seps, mz = seps;
    V Mxx = seps, Myy = seps, Mzz = seps, Mxy = seps, Mxz = seps, Myz = seps;
    V *const wbr = sbr + (size_t)warp * (NSLOT + 1) * NC * 32 + lane;   // [NSLOT + 1][NC][32]
    // one candidate at both cells: eps, and (acc) the u_s moments, and (b) the bracket
    auto visit = [&](const int k, V *b, const bool acc) {
        const T *rk = srec + k * RW;
        const Vec4<T> a = ld4<T>(rk);           // px, py, pz, r
        const Vec4<T> f = ld4<T>(rk + 4);       // f(r), Ux, Uy, Uz
        T dxa, dya, dza, dxb, dyb, dzb;
        cand_arm<L, T>(g, cxA, cyA, czA, a.x, a.y, a.z, dxa, dya, dza);
        cand_arm<L, T>(g, cxB, cyB, czB, a.x, a.y, a.z, dxb, dyb, dzb);
        const T ea = actA ? shell_eps<T>(dxa * dxa + dya * dya + dza * dza, a.w, f.x, ph.h) : (T)0;
        const T eb = actB ? shell_eps<T>(dxb * dxb + dyb * dyb + dzb * dzb, a.w, f.x, ph.h) : (T)0;
        if (ea > (T)0 || eb > (T)0) {
            const Vec4<T> o = ld4<T>(rk + 8);   // Ox, Oy, Oz, id
            const V dx = P::mk(dxa, dxb), dy = P::mk(dya, dyb), dz = P::mk(dza, dzb);
            // u_s = U + Omega x (x_n - X_p)
            const V usx = P::fma(P::sp(o.y), dz, P::fma(P::sp(-o.z), dy, P::sp(f.y)));
            const V usy = P::fma(P::sp(o.z), dx, P::fma(P::sp(-o.x), dz, P::sp(f.z)));
            const V usz = (L::D == 3) ? P::fma(P::sp(o.x), dy, P::fma(P::sp(-o.y), dx, P::sp(f.w))) : P::sp((T)0);
            // modified scheme weights by eps_s (normalised below); original by B(eps_s)
            const V e = P::mk(ea, eb);
            const V wgt = (PSC == 0) ? e
                                     : P::mk(ea * ph.tmh / (((T)1 - ea) + ph.tmh), eb * ph.tmh / (((T)1 - eb) + ph.tmh));
            if (acc) {
                seps = P::add(seps, wgt);
                mx = P::fma(wgt, usx, mx);
                my = P::fma(wgt, usy, my);
                const V wx = P::mul(wgt, usx), wy = P::mul(wgt, usy);
                Mxx = P::fma(wx, usx, Mxx);
                Myy = P::fma(wy, usy, Myy);
                Mxy = P::fma(wx, usy, Mxy);
                if (L::D == 3) {
                    mz = P::fma(wgt, usz, mz);
                    Mzz = P::fma(P::mul(wgt, usz), usz, Mzz);
                    Mxz = P::fma(wx, usz, Mxz);
                    Myz = P::fma(wy, usz, Myz);
                }
            }
            if (b) {
                const V s = (PSC == 0) ? e : P::mk(ea > (T)0 ? (T)1 : (T)0, eb > (T)0 ? (T)1 : (T)0);
                const V bx = P::mul(s, P::fma(rho, usx, px));
                const V by = P::mul(s, P::fma(rho, usy, py));
                if (L::D == 2) {
                    b[0] = bx; b[32] = by; b[64] = P::sub(P::mul(dx, by), P::mul(dy, bx));
                } else {
                    const V bz = P::mul(s, P::fma(rho, usz, pz));
                    b[0] = bx; b[32] = by; b[64] = bz;
                    b[96] = P::sub(P::mul(dy, bz), P::mul(dz, by));
                    b[128] = P::sub(P::mul(dz, bx), P::mul(dx, bz));
                    b[160] = P::sub(P::mul(dx, by), P::mul(dy, bx));
                }
            }
        } else if (b) {
#pragma unroll
            for (int c = 0; c < NC; ++c) b[32 * c] = P::sp((T)0);
        }
    };
    {
        unsigned mk = wmask;
        for (int js = 0; mk != 0u; ++js) {
            const int k = __ffs(mk) - 1;
            mk &= mk - 1u;
            visit(k, js < NSLOT ? wbr + js * NC * 32 : nullptr, true);
        }
    }

    // ---- weights (Eq. 8, 9, 13; Table 1 Step 5)
    const bool any_solid = __any_sync(kFull, seps.x > (T)0 || seps.y > (T)0);
    T BnA, cBA, BnB, cBB;
    psc_weights<PSC, T>(seps.x, ph.tmh, BnA, cBA);
    psc_weights<PSC, T>(seps.y, ph.tmh, BnB, cBB);
    const V Bn = P::mk(BnA, BnB), cB = P::mk(cBA, cBB);

    // ---- collision (Eq. 2-4, 10, 12), collected per cell:
    //      out_i = a1 d_i + B_n d_-i + w_i X_i,
    //      X_i = K0 + (e.u)(c2 + c4 e.u) + 3 rho e.m + 4.5 rho e.M.e + (1-B) guo (e.F)(3 + 9 e.u).
    //      Rows with no solid cell take the same code (B_n = 0 reduces it to BGK + Guo
    //      exactly): one copy of the collision keeps the kernel small enough for the
    //      instruction cache, which measured faster than a separate fluid branch.
    const V uu = P::fma(ux, ux, P::fma(uy, uy, P::mul(uz, uz)));
    const V uF = P::fma(ux, P::sp(ph.F[0]), P::fma(uy, P::sp(ph.F[1]), P::mul(uz, P::sp(ph.F[2]))));
    const V one = P::sp((T)1);
    {
        const V mxs = P::mul(cB, mx), mys = P::mul(cB, my), mzs = P::mul(cB, mz);
        const V omB = P::sub(one, Bn);
        const V oo = P::mul(omB, P::sp(ph.omega));
        const V a1 = P::sub(P::sub(one, oo), Bn);
        const V c1 = P::sub(oo, Bn);
        const V r3 = P::mul(P::sp((T)3), rho), r45 = P::mul(P::sp((T)4.5), rho);
        const V c2 = P::mul(r3, P::add(oo, Bn));
        const V c4 = P::mul(r45, c1);
        const V cg = P::mul(omB, P::sp(ph.guo));
        const V rc = P::mul(rho, cB);                      // the moments enter as c_B m, c_B M
        const V q15 = P::mul(P::sp((T)1.5), rc), q45 = P::mul(P::sp((T)4.5), rc), q90 = P::mul(P::sp((T)9), rc);
        const V trM = P::add(Mxx, P::add(Myy, Mzz));
        // K0 = c1 (drho - 1.5 rho uu) + B_n drho - 1.5 rho c_B tr M - 3 cg uF
        const V K0 = P::sub(P::fma(c1, P::sub(drho, P::mul(P::sp((T)1.5), P::mul(rho, uu))), P::mul(Bn, drho)),
                            P::fma(q15, trM, P::mul(P::mul(P::sp((T)3), cg), uF)));
        const V m3x = P::mul(r3, mxs), m3y = P::mul(r3, mys), m3z = P::mul(r3, mzs);
        const V Axx = P::mul(q45, Mxx), Ayy = P::mul(q45, Myy), Azz = P::mul(q45, Mzz);
        const V Axy = P::mul(q90, Mxy), Axz = P::mul(q90, Mxz), Ayz = P::mul(q90, Myz);   // 2 x 4.5 rho c_B M_ab
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int o = opp<L>(i);
            const int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
            const T w = (T)weight<L>(i);
            V X = K0;
            if (ex || ey || ez) {
                const V eu = edot2<L, T>(i, ux, uy, uz);
                const V em = edot2<L, T>(i, m3x, m3y, m3z);
                const T eF = edot<L, T>(i, ph.F[0], ph.F[1], ph.F[2]);
                V eMe = P::sp((T)0);
                bool first = true;
                auto addm = [&](V v, bool neg) {
                    if (first) { eMe = neg ? P::sub(P::sp((T)0), v) : v; first = false; }
                    else eMe = neg ? P::sub(eMe, v) : P::add(eMe, v);
                };
                if (ex) addm(Axx, false);
                if (ey) addm(Ayy, false);
                if (L::D == 3 && ez) addm(Azz, false);
                if (ex && ey) addm(Axy, ex != ey);
                if (ex && ez) addm(Axz, ex != ez);
                if (ey && ez) addm(Ayz, ey != ez);
                // eu (c2 + c4 eu) + em + eMe + cg eF (3 + 9 eu)
                V t = P::fma(eu, P::fma(c4, eu, c2), P::add(em, eMe));
                t = P::fma(P::mul(cg, P::sp(eF)), P::fma(P::sp((T)9), eu, P::sp((T)3)), t);
                X = P::add(X, t);
            }
            const V out = P::fma(a1, df[i], P::fma(Bn, df[o], P::mul(P::sp(w * ssc), X)));
            store_pair<S>(fout, (long long)i * N + cellA, (long long)i * N + cellB, out.x, out.y, actA, actB,
                          L::Q * N);
        }
    }

    // ---- force and torque (Eq. 14; Eq. 11 original): per candidate the warp's sum over both
    //      cells of mult * bracket with mult = c_B (B_n), one shared-memory partial per warp
    if (lane == 0) s_mask[warp] = any_solid ? wmask : 0u;
    if (any_solid) {
        const V mult = (PSC == 0) ? cB : Bn;
        constexpr int NCP = (NC <= 4) ? 4 : 8;
        const int cs = lane >> ((NCP == 4) ? 3 : 2);
        unsigned mf = wmask;
        auto reduce_store = [&](const int k, const V *b, const int stride) {
            T v[NCP];
#pragma unroll
            for (int c = 0; c < NCP; ++c) {
                if (c < NC) {
                    const V m = P::mul(mult, b[c * stride]);
                    v[c] = m.x + m.y;
                } else {
                    v[c] = (T)0;
                }
            }
            const T tot = warp_sum_spread<NCP>(v, lane);
            if ((lane & (32 / NCP - 1)) == 0 && cs < NC) part[(warp * kPairCap + k) * NC + cs] = tot;
        };
        // the first NSLOT candidates' brackets are kept; further ones are evaluated again
        // (brackets only) into the scratch slot
        V *const scratch = wbr + NSLOT * NC * 32;
        for (int js = 0; mf != 0u; ++js) {
            const int k = __ffs(mf) - 1;
            mf &= mf - 1u;
            if (js >= NSLOT) visit(k, scratch, false);
            reduce_store(k, js < NSLOT ? wbr + js * NC * 32 : scratch, 32);
        }
    }
}

// One plain-fluid tile with two cells per thread (rows as in the particle-tile path): BGK +
// Guo + pull on FP32 pairs. With F = 0 the Guo terms add exact zeros, so HASF = true gives
// the same results as HASF = false.
template <class L, typename S, bool HASF>
__device__ __forceinline__ void fluid_tile_pair(const S *__restrict__ fin, S *__restrict__ fout, const Geom &g,
                                                const PhysT<typename Store<S>::T> &ph, const int x0, const int y0,
                                                const int z0, int *flags) {
    using T = typename Store<S>::T;
    using P = Pr<T>;
    using V = typename P::V;
    constexpr int Q = L::Q;
    const long long N = g.ncell;
    const int lane = threadIdx.x, warp = threadIdx.y;
    const PairCells<L> pc(lane, warp);
    const int xA = x0 + pc.xA, xB = x0 + pc.xB;
    const int yA = y0 + pc.yA, yB = y0 + pc.yB, zA = z0 + pc.zA, zB = z0 + pc.zB;
    const bool actA = cell_active<L>(g, xA, yA, zA);
    const bool actB = cell_active<L>(g, xB, yB, zB);
    const long long cellA = xA + (long long)g.n[0] * (yA + (long long)g.n[1] * zA);
    const long long cellB = xB + (long long)g.n[0] * (yB + (long long)g.n[1] * zB);
    const bool interior = x0 >= 1 && x0 + L::TX < g.n[0] && y0 >= 1 && y0 + L::TY < g.n[1] &&
                          (L::D == 2 || (z0 >= 1 && z0 + L::TZ < g.n[2]));
    constexpr bool SC = Store<S>::kScaled;   // as in psc_tile_pair: scale folded in
    T da[Q], db[Q];
    pull_pair<L, S>(fin, g, ph, interior, xA, xB, yA, yB, zA, zB, cellA, cellB, actA, actB, da, db);
    V df[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) df[i] = P::mk(da[i], db[i]);
    V drho = df[0], jx = P::sp((T)0), jy = P::sp((T)0), jz = P::sp((T)0);
#pragma unroll
    for (int i = 1; i < Q; ++i) drho = P::add(drho, df[i]);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (L::ex(i)) jx = L::ex(i) > 0 ? P::add(jx, df[i]) : P::sub(jx, df[i]);
        if (L::ey(i)) jy = L::ey(i) > 0 ? P::add(jy, df[i]) : P::sub(jy, df[i]);
        if (L::ez(i)) jz = L::ez(i) > 0 ? P::add(jz, df[i]) : P::sub(jz, df[i]);
    }
    const T ssc = SC ? (T)ph.sc.x : (T)1;
    if (SC) {
        const V is = P::sp((T)ph.sc.y);
        drho = P::mul(drho, is); jx = P::mul(jx, is); jy = P::mul(jy, is); jz = P::mul(jz, is);
    }
    const V rho = P::add(P::sp((T)1), drho);
    const V irho = P::mk((T)1 / rho.x, (T)1 / rho.y);
    V ux, uy, uz;
    if (HASF) {
        ux = P::mul(P::add(jx, P::sp((T)0.5 * ph.F[0])), irho);
        uy = P::mul(P::add(jy, P::sp((T)0.5 * ph.F[1])), irho);
        uz = P::mul(P::add(jz, P::sp((T)0.5 * ph.F[2])), irho);
    } else {
        ux = P::mul(jx, irho); uy = P::mul(jy, irho); uz = P::mul(jz, irho);
    }
    if ((actA && !(rho.x > (T)0)) || (actB && !(rho.y > (T)0))) atomicOr(flags, 1);
    const V uu = P::fma(ux, ux, P::fma(uy, uy, P::mul(uz, uz)));
    const V base_eq = P::sub(drho, P::mul(P::sp((T)1.5), P::mul(rho, uu)));
    const V om1 = P::sp((T)1 - ph.omega), om = P::sp(ph.omega);
    V guo3uF = P::sp((T)0);
    if (HASF) {
        const V uF = P::fma(ux, P::sp(ph.F[0]), P::fma(uy, P::sp(ph.F[1]), P::mul(uz, P::sp(ph.F[2]))));
        guo3uF = P::mul(P::sp((T)3 * ph.guo), uF);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T w = (T)weight<L>(i) * ssc;
        const V eu = edot2<L, T>(i, ux, uy, uz);
        // w (base_eq + rho eu (3 + 4.5 eu))
        const V dfeq = P::mul(P::sp(w), P::fma(P::mul(rho, eu), P::fma(P::sp((T)4.5), eu, P::sp((T)3)), base_eq));
        V out = P::fma(om1, df[i], P::mul(om, dfeq));
        if (HASF) {
            const T eF = edot<L, T>(i, ph.F[0], ph.F[1], ph.F[2]);
            out = P::add(out, P::mul(P::sp(w), P::sub(P::fma(P::sp((T)9 * ph.guo * eF), eu, P::sp((T)3 * ph.guo * eF)), guo3uF)));
        }
        store_pair<S>(fout, (long long)i * N + cellA, (long long)i * N + cellB, out.x, out.y, actA, actB,
                          L::Q * N);
    }
}

// The particle-tile kernel: a persistent grid takes tiles with candidates from the compact
// list through a work counter (tiles differ in cost, so the counter balances the SMs; the
// next tile's index is fetched while the current one runs). With STEAL it then takes the
// tiles without candidates the same way, so one launch covers the lattice and its blocks
// share out the end of the step. Tiles with more than kPairCap candidates are left to
// k_collide_overflow, which also clears the counters for the next launch.
template <class L, typename S, int PSC, bool STEAL>
__global__ void __launch_bounds__(kPThreads, (sizeof(typename Store<S>::T) == 8) ? 2 : ((L::Q == 9) ? 6 : 4))
k_collide_stream(const S *__restrict__ fin, S *__restrict__ fout, Geom g,
                 PhysT<typename Store<S>::T> ph, Tiles tl, Parts pd, int *flags) {
    using T = typename Store<S>::T;
    using V = typename Pr<T>::V;
    constexpr int NC = (L::D == 2) ? 3 : 6;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_mask[2][kPWarps];
    __shared__ int s_next[2];
    T *const sm = reinterpret_cast<T *>(smem);
    constexpr int rsz = kPairCap * RW, psz = kPWarps * kPairCap * NC;
    V *const sbr = reinterpret_cast<V *>(sm + 2 * (rsz + psz));
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int npsc = tl.stats[4];
    const int limit = min(tl.cap, kPairCap);
    if (tid == 0) s_next[0] = atomicAdd(&tl.stats[6], 1);
    __syncthreads();
    const T *blocks = reinterpret_cast<const T *>(tl.blocks);
    int buf = 0, prev_cnt = 0;
    const T *prev_recs = blocks;
    for (;;) {
        const int it = s_next[buf];
        if (it >= npsc) break;
        if (tid == 0) s_next[buf ^ 1] = atomicAdd(&tl.stats[6], 1);
        const uint2 ent = tl.order[it];
        const int cnt = tl.count[ent.x];
        const T *recs = blocks + (size_t)ent.x * block_elems<T>(tl.cap) + head_elems<T>();
        T *const cur_part = sm + 2 * rsz + buf * psz;
        T *const prv_part = sm + 2 * rsz + (buf ^ 1) * psz;
        if (cnt <= limit) {
            psc_tile_pair<L, S, PSC>(ent, cnt, fin, fout, g, ph, tl, pd, flags, sm + buf * rsz, cur_part, s_mask[buf],
                                     prev_cnt, prev_recs, prv_part, s_mask[buf ^ 1], sbr);
            prev_cnt = cnt;
        } else {
            __syncthreads();
            pair_flush<L, T>(prev_cnt, prev_recs, prv_part, s_mask[buf ^ 1], pd, tid);
            prev_cnt = 0;
        }
        prev_recs = recs;
        buf ^= 1;
    }
    __syncthreads();
    pair_flush<L, T>(prev_cnt, prev_recs, sm + 2 * rsz + (buf ^ 1) * psz, s_mask[buf ^ 1], pd, tid);
    if (STEAL) {
        const long long ntiles = (long long)g.nt[0] * g.nt[1] * g.nt[2];
        const int nfl = tl.stats[5];
        const uint2 *const flist = tl.order + ntiles;
        __syncthreads();
        if (tid == 0) s_next[0] = atomicAdd(&tl.stats[3], 1);
        __syncthreads();
        buf = 0;
        for (;;) {
            const int it = s_next[buf];
            if (it >= nfl) break;
            if (tid == 0) s_next[buf ^ 1] = atomicAdd(&tl.stats[3], 1);
            const uint2 ent = flist[it];
            const unsigned ty = ent.y & 0xffffu, tz = ent.y >> 16;
            fluid_tile_pair<L, S, true>(fin, fout, g, ph,
                                        (int)(ent.x - (unsigned)g.nt[0] * (ty + (unsigned)g.nt[1] * tz)) * L::TX,
                                        (int)ty * L::TY, (int)tz * L::TZ, flags);
            __syncthreads();     // the next index is visible, this one may be overwritten
            buf ^= 1;
        }
    }
}

// Plain-fluid tiles: without particles one block per tile; with particles a persistent
// grid striding over the list of tiles without candidates (beside the particle-tile kernel).
template <class L, typename S, bool HASF>
__global__ void __launch_bounds__(kPThreads, (L::Q == 9) ? 8 : 5)
k_fluid_pair(const S *__restrict__ fin, S *__restrict__ fout, Geom g, PhysT<typename Store<S>::T> ph, Tiles tl,
             int np, int *flags) {
    if (np == 0) {
        fluid_tile_pair<L, S, HASF>(fin, fout, g, ph, blockIdx.x * L::TX, blockIdx.y * L::TY, blockIdx.z * L::TZ,
                                    flags);
        return;
    }
    const long long ntiles = (long long)g.nt[0] * g.nt[1] * g.nt[2];
    const int nfl = tl.stats[5];
    const uint2 *const flist = tl.order + ntiles;
    for (int it = blockIdx.x; it < nfl; it += gridDim.x) {
        const uint2 ent = flist[it];
        const unsigned ty = ent.y & 0xffffu, tz = ent.y >> 16;
        fluid_tile_pair<L, S, HASF>(fin, fout, g, ph, (int)(ent.x - (unsigned)g.nt[0] * (ty + (unsigned)g.nt[1] * tz)) * L::TX,
                                    (int)ty * L::TY, (int)tz * L::TZ, flags);
    }
}
