// o2pic_push.cu -- the fused per-step particle kernel of libo2pic.
//
// One launch advances every live superparticle of every discharge by one time
// step (paper Sec. II (i) and Sec. III):
//   gather E at x^n (linear interpolation from a shared-memory copy of the
//   node field) -> leapfrog v^{n+1/2}, x^{n+1} -> absorption at x < 0 or
//   x >= L -> null-collision test against nu_max (one Philox4x32-10 block
//   serves four consecutive slots) -> for candidates, a gas molecule from the
//   Maxwellian at T, channel walk over sum_j n_j sigma_j(E) u and the
//   kinematics of the chosen reaction -> births staged per chunk and appended
//   in parent order through a decoupled look-back over chunks -> linear
//   charge assignment of x^{n+1} into a per-block shared-memory grid (warp
//   aggregated, exact fixed point in the FP32 path), flushed to the global
//   accumulators with one atomic per touched node.
//
// Particles are SoA with the position as (int32 cell, offset in [0,1)) and
// velocities in cells per step.  Slots are processed in chunks of 1024
// (256 threads x 4 consecutive slots, 16-byte vector loads), handed out in
// increasing order by an atomic ticket to a persistent grid.
#include <cstdio>

#include "o2pic_launch.h"

namespace o2 {

template <typename Real> struct AccT;
template <> struct AccT<float> { using T = unsigned long long; };
template <> struct AccT<double> { using T = double; };

template <typename Real> struct Lut;
template <> struct Lut<float> {
    static __device__ __forceinline__ const float *E(const WsPtrs &W) { return W.lutEf; }
    static __device__ __forceinline__ const float *S(const WsPtrs &W) { return W.lutSf; }
};
template <> struct Lut<double> {
    static __device__ __forceinline__ const double *E(const WsPtrs &W) { return W.lutE; }
    static __device__ __forceinline__ const double *S(const WsPtrs &W) { return W.lutS; }
};

__device__ __forceinline__ void ld4(const int *p, int v[4])
{
    int4 t = *reinterpret_cast<const int4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void st4(int *p, const int v[4])
{
    *reinterpret_cast<int4 *>(p) = make_int4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void ld4(const float *p, float v[4])
{
    float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void st4(float *p, const float v[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void ld4(const double *p, double v[4])
{
    double2 a = reinterpret_cast<const double2 *>(p)[0];
    double2 b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(double *p, const double v[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Interpolation of the gas-channel cross sections of one projectile at the
// centre-of-mass energy E [eV]: piecewise linear in E on the shared geometric
// grid, end values held outside it, zero below each channel's threshold.
template <typename Real>
struct XsPoint {
    int k;       // segment
    Real f;      // fraction inside the segment
    int region;  // 0 below the grid, 1 inside, 2 above
};

template <typename Real>
__device__ __forceinline__ XsPoint<Real> xs_locate(const TableDesc &T, const Real *lutE, Real E)
{
    XsPoint<Real> p;
    const Real *nodes = lutE + T.off;
    const int n = T.n;
    if (!(E > nodes[0])) {
        p.region = 0; p.k = 0; p.f = Real(0);
        return p;
    }
    if (E >= nodes[n - 1]) {
        p.region = 2; p.k = n - 2; p.f = Real(1);
        return p;
    }
    Real t = (log(E) - Real(T.lnE0)) * Real(T.inv_dlog);
    int k = (int)t;
    k = k < 0 ? 0 : (k > n - 2 ? n - 2 : k);
    // the logarithm only guesses the segment; the node comparison decides
    while (k > 0 && E < nodes[k]) --k;
    while (k < n - 2 && E >= nodes[k + 1]) ++k;
    p.region = 1;
    p.k = k;
    p.f = (E - nodes[k]) / (nodes[k + 1] - nodes[k]);
    return p;
}

template <typename Real>
__device__ __forceinline__ Real xs_value(const TableDesc &T, const Real *lutS,
                                         const XsPoint<Real> &p, Real E)
{
    if (E < Real(T.th)) return Real(0);
    const Real *s = lutS + T.off;
    if (p.region == 0) return s[0];
    if (p.region == 2) return s[T.n - 1];
    Real a = s[p.k], b = s[p.k + 1];
    return a + p.f * (b - a);
}

// centre-of-mass binary collision in normalised units: relative speed
// sqrt(u^2 - dloss) along n (Eq. 5 with dloss = 2 dE/mu (dt/dx)^2)
template <typename Real>
__device__ __forceinline__ void cm_scatter(Real mfrac, Real Mfrac, const Real v[3],
                                           const Real V[3], Real dloss, const Real n[3],
                                           Real vo[3], Real Vo[3])
{
    Real g0 = v[0] - V[0], g1 = v[1] - V[1], g2 = v[2] - V[2];
    Real u2 = g0 * g0 + g1 * g1 + g2 * g2 - dloss;
    Real up = u2 > Real(0) ? sqrt(u2) : Real(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        Real vcm = mfrac * v[q] + Mfrac * V[q];
        vo[q] = vcm + Mfrac * up * n[q];
        Vo[q] = vcm - mfrac * up * n[q];
    }
}

template <typename Real>
__device__ __forceinline__ void ee_elastic(Real a[3], Real b[3], const Real n[3])
{
    Real g0 = a[0] - b[0], g1 = a[1] - b[1], g2 = a[2] - b[2];
    Real u = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        Real c = Real(0.5) * (a[q] + b[q]);
        a[q] = c + Real(0.5) * u * n[q];
        b[q] = c - Real(0.5) * u * n[q];
    }
}

template <typename Real>
struct BirthStage {
    int *cell, *tag;
    Real *off, *vx, *vy, *vz;
    int *nb;
};

template <typename Real>
__device__ __forceinline__ void stage_birth(const BirthStage<Real> &B, Ctl *ctl, int tag,
                                            int sp, int c, Real off, const Real v[3])
{
    int pos = atomicAdd(B.nb, 1);
    if (pos >= BIRTH_CAP) {
        set_status(ctl, ST_BIRTHBUF);
        return;
    }
    B.cell[pos] = c;
    B.tag[pos] = (tag << 2) | sp;
    B.off[pos] = off;
    B.vx[pos] = v[0];
    B.vy[pos] = v[1];
    B.vz[pos] = v[2];
}

// One gas-target candidate (null-collision method).  Returns false if the
// particle died.  v is updated in place; products are staged.
template <typename Real>
__device__ __noinline__ bool gas_collide(const WsPtrs &W, const Disc &Dd, int s, unsigned idx,
                                         unsigned long long step, Real &vx, Real &vy, Real &vz,
                                         int c, Real off, int tag, const BirthStage<Real> &B,
                                         unsigned *s_cnt)
{
    const SpeciesC &S = Dd.sp[s];
    const Real *lutE = Lut<Real>::E(W);
    const Real *lutS = Lut<Real>::S(W);
    uint4 a = rng_block(Dd.seed, Dd.discharge, s, 1, 0, 0, step, idx);
    uint4 b = rng_block(Dd.seed, Dd.discharge, s, 1, 0, 1, step, idx);
    Real n0, n1, n2, n3;
    box_muller<Real>(a.x, a.y, n0, n1);
    box_muller<Real>(a.z, a.w, n2, n3);
    const Real vg = Real(S.vgas_n);
    Real V[3] = {vg * n0, vg * n1, vg * n2};
    Real v[3] = {vx, vy, vz};
    Real g0 = v[0] - V[0], g1 = v[1] - V[1], g2 = v[2] - V[2];
    Real u2 = g0 * g0 + g1 * g1 + g2 * g2;
    Real u = sqrt(u2);
    Real E = Real(S.Ek) * u2;
    Real target = unif<Real>(b.x) * Real(S.numax_n);
    const TableDesc &T0 = W.tables[S.table_lo];
    XsPoint<Real> pt = xs_locate<Real>(T0, lutE, E);
    Real cum = Real(0);
    int chosen = -1;
    for (int j = 0; j < S.nch; ++j) {
        const GasChan &ch = S.ch[j];
        Real sg = xs_value<Real>(W.tables[ch.table], lutS, pt, E);
        cum += Real(ch.coef) * sg * u;
        if (chosen < 0 && target < cum) chosen = j;
    }
    if (cum > Real(S.numax_n)) atomicAdd(&s_cnt[C_VIOL_GAS], 1u);
    if (chosen < 0) return true;  // null event
    const GasChan &ch = S.ch[chosen];
    const int r = ch.reaction;
    atomicAdd(&s_cnt[C_EVENTS + r], 1u);
    Real nd[3];
    iso_dir<Real>(unif<Real>(b.y), unif<Real>(b.z), nd);
    const Real mf = Real(S.mfrac), Mf = Real(S.Mfrac);
    Real vo[3], Vo[3];
    switch (r) {
    case 4: case 5:
        cm_scatter<Real>(mf, Mf, v, V, Real(0), nd, vo, Vo);
        vx = vo[0]; vy = vo[1]; vz = vo[2];
        return true;
    case 6:
        if (Dd.cx_iso) {
            cm_scatter<Real>(mf, Mf, v, V, Real(0), nd, vo, Vo);
            vx = vo[0]; vy = vo[1]; vz = vo[2];
        } else {
            vx = V[0]; vy = V[1]; vz = V[2];  // resonant exchange
        }
        return true;
    case 15: {
        const TableDesc &Tc = W.tables[ch.table];
        Real Ea = E - Real(Tc.th);
        Ea = Ea > Real(0) ? Ea : Real(0);
        Real w = sqrt(Ea * Real(Dd.f15));
        Real pv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) pv[q] = mf * v[q] + Mf * V[q] + w * nd[q];
        stage_birth<Real>(B, W.ctl, tag, 1, c, off, pv);
        return false;
    }
    case 16: {
        Real sp = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * Real(Dd.f16);
        Real pv[3] = {sp * nd[0], sp * nd[1], sp * nd[2]};
        stage_birth<Real>(B, W.ctl, tag, 0, c, off, pv);
        return false;
    }
    case 17: {
        Real w = sqrt(E * Real(Dd.f17));
        Real pv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) pv[q] = mf * v[q] + Mf * V[q] + w * nd[q];
        stage_birth<Real>(B, W.ctl, tag, 0, c, off, pv);
        return false;
    }
    case 18: {
        cm_scatter<Real>(mf, Mf, v, V, Real(ch.dloss), nd, vo, Vo);
        uint4 e = rng_block(Dd.seed, Dd.discharge, s, 1, 0, 2, step, idx);
        Real n2v[3];
        iso_dir<Real>(unif<Real>(e.x), unif<Real>(e.y), n2v);
        Real e2[3] = {Vo[0], Vo[1], Vo[2]};
        ee_elastic<Real>(vo, e2, n2v);
        vx = vo[0]; vy = vo[1]; vz = vo[2];
        stage_birth<Real>(B, W.ctl, tag, 0, c, off, e2);
        stage_birth<Real>(B, W.ctl, tag | 1, 2, c, off, Vo);
        return true;
    }
    default:  // 7-12: inelastic, Eq. 5
        cm_scatter<Real>(mf, Mf, v, V, Real(ch.dloss), nd, vo, Vo);
        vx = vo[0]; vy = vo[1]; vz = vo[2];
        return true;
    }
}

template <typename Acc> __device__ __forceinline__ void acc_add(Acc *a, Acc v);
template <> __device__ __forceinline__ void acc_add(unsigned long long *a, unsigned long long v)
{
    atomicAdd(a, v);
}
template <> __device__ __forceinline__ void acc_add(double *a, double v) { atomicAdd(a, v); }

// deposit of one slot per lane, aggregated over lanes that share a cell
__device__ __forceinline__ void deposit_warp(unsigned long long *sAcc, int c, float off)
{
    unsigned w1 = 0, w0 = 0;
    if (c >= 0) {
        w1 = __float2uint_rn(off * (float)(1 << FIX_BITS));
        w0 = (1u << FIX_BITS) - w1;
    }
    unsigned peers = __match_any_sync(0xffffffffu, c);
    unsigned s0 = __reduce_add_sync(peers, w0);
    unsigned s1 = __reduce_add_sync(peers, w1);
    if (c >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) {
        atomicAdd(&sAcc[c], (unsigned long long)s0);
        atomicAdd(&sAcc[c + 1], (unsigned long long)s1);
    }
}
__device__ __forceinline__ void deposit_warp(double *sAcc, int c, double off)
{
    if (c >= 0) {
        atomicAdd(&sAcc[c], 1.0 - off);
        atomicAdd(&sAcc[c + 1], off);
    }
}

// charge of one particle added to (sign > 0) or removed from the global
// accumulator of its species (births, pair-pass kills)
__device__ __forceinline__ void deposit_global(unsigned long long *acc, int c, float off, int sign)
{
    unsigned w1 = __float2uint_rn(off * (float)(1 << FIX_BITS));
    unsigned w0 = (1u << FIX_BITS) - w1;
    unsigned long long a = w0, b = w1;
    if (sign < 0) { a = 0ull - a; b = 0ull - b; }
    atomicAdd(&acc[c], a);
    atomicAdd(&acc[c + 1], b);
}
__device__ __forceinline__ void deposit_global(double *acc, int c, double off, int sign)
{
    atomicAdd(&acc[c], sign * (1.0 - off));
    atomicAdd(&acc[c + 1], sign * off);
}

template <typename Real> __device__ __forceinline__ typename AccT<Real>::T *acc_global(const WsPtrs &W);
template <> __device__ __forceinline__ unsigned long long *acc_global<float>(const WsPtrs &W) { return W.acc_fix; }
template <> __device__ __forceinline__ double *acc_global<double>(const WsPtrs &W) { return W.acc_dbl; }

template <typename Real, bool DIAG>
__global__ void __launch_bounds__(PUSH_THREADS)
k_push(WsPtrs W, Pools<Real> P, int par, int Nmax, int eedf_max, int fm_max)
{
    using Acc = typename AccT<Real>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    Acc *sAcc = reinterpret_cast<Acc *>(smem);
    Real *sE = reinterpret_cast<Real *>(sAcc + (Nmax + 2));
    Real *bOff = sE + (Nmax + 2);
    Real *bVx = bOff + BIRTH_CAP;
    Real *bVy = bVx + BIRTH_CAP;
    Real *bVz = bVy + BIRTH_CAP;
    int *bCell = reinterpret_cast<int *>(bVz + BIRTH_CAP);
    int *bTag = bCell + BIRTH_CAP;
    int *bRank = bTag + BIRTH_CAP;
    unsigned *sEedf = reinterpret_cast<unsigned *>(bRank + BIRTH_CAP);
    unsigned *sFm = sEedf + eedf_max;

    __shared__ int s_ticket, s_nb;
    __shared__ int s_bc[NSP], s_bx[NSP];
    __shared__ unsigned s_cnt[C_NCOUNT];

    Ctl *ctl = W.ctl;
    const int cur = ctl->cur;
    const unsigned long long step = ctl->step[par];
    const int total = ctl->total_chunks;
    const int nds = W.D * NSP;
    int *cellA = P.cell[cur];
    Real *offA = P.off[cur], *vxA = P.vx[cur], *vyA = P.vy[cur], *vzA = P.vz[cur];
    Acc *accG = acc_global<Real>(W);
    const int tid = threadIdx.x;
    BirthStage<Real> B{bCell, bTag, bOff, bVx, bVy, bVz, &s_nb};

    int ds = -1, d = -1;
    for (int q = tid; q < C_NCOUNT; q += PUSH_THREADS) s_cnt[q] = 0;

    auto flush = [&](int fds) {
        const int fd = fds / NSP, fs = fds % NSP;
        const Disc &Dd = W.disc[fd];
        __syncthreads();
        Acc *g = accG + (size_t)fs * W.total_nodes + Dd.gbase;
        for (int i = tid; i <= Dd.N; i += PUSH_THREADS) {
            Acc v = sAcc[i];
            if (v != Acc(0)) acc_add(&g[i], v);
        }
        for (int q = tid; q < C_NCOUNT; q += PUSH_THREADS) {
            if (s_cnt[q]) atomicAdd(&W.counters[(size_t)fd * C_NCOUNT + q], (unsigned long long)s_cnt[q]);
        }
        if (DIAG) {
            if (fs == 0)
                for (int i = tid; i < Dd.eedf_bins; i += PUSH_THREADS)
                    if (sEedf[i]) atomicAdd(&W.eedf[Dd.eedf_base + i], sEedf[i]);
            if (fs == 1)
                for (int i = tid; i < Dd.fm_bins * Dd.fm_xbins; i += PUSH_THREADS)
                    if (sFm[i]) atomicAdd(&W.fm[Dd.fm_base + i], sFm[i]);
        }
        __syncthreads();
    };

    for (;;) {
        if (tid == 0) {
            s_ticket = (int)atomicAdd(&ctl->ticket, 1u);
            s_nb = 0;
        }
        if (tid < NSP) s_bc[tid] = 0;
        __syncthreads();
        const int t = s_ticket;
        if (t >= total) break;
        int nx = ds < 0 ? 0 : ds;
        while (nx < nds && !(t >= W.cnt[nx].chunk0 && t < W.cnt[nx].chunk0 + W.cnt[nx].nchunk)) ++nx;
        if (nx >= nds) {  // cannot happen with a consistent chunk table
            if (tid == 0) set_status(ctl, ST_BADSTATE);
            break;
        }
        if (nx != ds) {
            if (ds >= 0) flush(ds);
            const int nd = nx / NSP;
            const Disc &Dn = W.disc[nd];
            if (nd != d) {
                const Real *Eg = reinterpret_cast<const Real *>(W.Ereal) + Dn.gbase;
                for (int i = tid; i <= Dn.N; i += PUSH_THREADS) sE[i] = Eg[i];
                d = nd;
            }
            for (int i = tid; i <= Dn.N + 1; i += PUSH_THREADS) sAcc[i] = Acc(0);
            for (int q = tid; q < C_NCOUNT; q += PUSH_THREADS) s_cnt[q] = 0;
            if (DIAG) {
                for (int i = tid; i < eedf_max; i += PUSH_THREADS) sEedf[i] = 0;
                for (int i = tid; i < fm_max; i += PUSH_THREADS) sFm[i] = 0;
            }
            ds = nx;
            __syncthreads();
        }
        const int s = ds % NSP;
        const Disc &Dd = W.disc[d];
        const SpeciesC &S = Dd.sp[s];
        const Counts &C = W.cnt[ds];
        const int N = Dd.N;
        const int pb = Dd.pbase[s];
        const int base = pb + (t - C.chunk0) * CHUNK;
        const int end = pb + C.n_snap;
        const int i0 = base + 4 * tid;
        const Real qm = Real(S.qm);

        int c[4];
        Real off[4], vx[4];
        const bool full = i0 + 3 < end;
        if (full) {
            ld4(cellA + i0, c);
            ld4(offA + i0, off);
            ld4(vxA + i0, vx);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool in = i0 + k < end;
                c[k] = in ? cellA[i0 + k] : -2;
                off[k] = in ? offA[i0 + k] : Real(0);
                vx[k] = in ? vxA[i0 + k] : Real(0);
            }
        }
        uint4 w4 = make_uint4(0, 0, 0, 0);
        if (c[0] >= 0 || c[1] >= 0 || c[2] >= 0 || c[3] >= 0)
            w4 = rng_block(Dd.seed, Dd.discharge, s, 0, 0, 0, step, (unsigned)((i0 - pb) >> 2));
        const unsigned wk[4] = {w4.x, w4.y, w4.z, w4.w};
        unsigned nslots = 0, ncand = 0;

#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int ck = c[k];
            int dep = -1;
            if (ck >= -1) ++nslots;
            if (ck >= 0) {
                const Real e0 = sE[ck], e1 = sE[ck + 1];
                const Real ep = e0 + off[k] * (e1 - e0);
                Real v = vx[k] + qm * ep;
                Real o = off[k] + v;
                Real fl = floor(o);
                bool bad = !(fl > Real(-2 * N - 4) && fl < Real(2 * N + 4));
                int cn = bad ? (v < Real(0) ? -1 : N) : ck + (int)fl;
                o -= fl;
                if (o >= Real(1)) { o -= Real(1); cn += 1; }
                vx[k] = v;
                if (cn < 0 || cn >= N) {
                    const int wall = cn < 0 ? 0 : 1;
                    atomicAdd(&s_cnt[C_ABS + 2 * s + wall], 1u);
                    if (s == 2 && Dd.iedf_bins > 0) {
                        Real vy = vyA[i0 + k], vz = vzA[i0 + k];
                        Real Ei = Real(S.ke_eV) * (v * v + vy * vy + vz * vz);
                        Real bb = floor(Ei * Real(Dd.iedf_scale));
                        if (bb >= Real(0) && bb < Real(Dd.iedf_bins))
                            atomicAdd(&W.iedf[Dd.iedf_base + wall * Dd.iedf_bins + (int)bb], 1u);
                    }
                    c[k] = -1;
                } else {
                    off[k] = o;
                    c[k] = cn;
                    bool alive = true;
                    Real vy = Real(0), vz = Real(0);
                    bool have_v = false;
                    if (wk[k] < S.tnull) {
                        ++ncand;
                        vy = vyA[i0 + k];
                        vz = vzA[i0 + k];
                        have_v = true;
                        Real ux = vx[k];
                        alive = gas_collide<Real>(W, Dd, s, (unsigned)(i0 + k - pb), step, ux, vy, vz,
                                                  cn, o, ((tid << 2) | k) << 1, B, s_cnt);
                        if (alive) {
                            vx[k] = ux;
                            vyA[i0 + k] = vy;
                            vzA[i0 + k] = vz;
                        } else {
                            c[k] = -1;
                        }
                    }
                    if (alive) {
                        dep = cn;
                        if (DIAG) {
                            if (s == 0 && cn == N / 2 && Dd.eedf_bins > 0) {
                                if (!have_v) { vy = vyA[i0 + k]; vz = vzA[i0 + k]; }
                                Real Ee = Real(S.ke_eV) * (vx[k] * vx[k] + vy * vy + vz * vz);
                                Real bb = floor(Ee * Real(Dd.eedf_scale));
                                if (bb >= Real(0) && bb < Real(Dd.eedf_bins)) atomicAdd(&sEedf[(int)bb], 1u);
                            }
                            if (s == 1 && Dd.fm_bins > 0) {
                                Real Es = Real(S.ke_eV) * vx[k] * vx[k];
                                if (vx[k] < Real(0)) Es = -Es;
                                Real bb = floor((Es + Real(Dd.fm_emax)) * Real(Dd.fm_scale));
                                if (bb >= Real(0) && bb < Real(Dd.fm_bins)) {
                                    int xb = (int)(((long long)cn * Dd.fm_xbins) / N);
                                    atomicAdd(&sFm[xb * Dd.fm_bins + (int)bb], 1u);
                                }
                            }
                        }
                    }
                }
            }
            deposit_warp(sAcc, dep, off[k]);
        }
        if (nslots) atomicAdd(&s_cnt[C_SLOTS], nslots);
        if (ncand) atomicAdd(&s_cnt[C_CANDS], ncand);
        if (full) {
            st4(cellA + i0, c);
            st4(offA + i0, off);
            st4(vxA + i0, vx);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (i0 + k < end) {
                    cellA[i0 + k] = c[k];
                    offA[i0 + k] = off[k];
                    vxA[i0 + k] = vx[k];
                }
            }
        }
        __syncthreads();

        // ---- births: order within the chunk by (slot, product), then the
        // decoupled look-back gives this chunk's place among all chunks of
        // its discharge (chunks are numbered in (species, slot) order).
        const int nb = s_nb < BIRTH_CAP ? s_nb : BIRTH_CAP;
        for (int r = tid; r < nb; r += PUSH_THREADS) {
            const int tg = bTag[r];
            const int sp = tg & 3;
            int rank = 0;
            for (int q = 0; q < nb; ++q) {
                const int tq = bTag[q];
                rank += ((tq & 3) == sp) && (tq < tg);
            }
            bRank[r] = rank;
            atomicAdd(&s_bc[sp], 1);
        }
        __syncthreads();
        if (tid < NSP) {
            const int sp = tid;
            const unsigned long long epoch = (step + 1ull) & 0xFFFFFFFFull;
            const int first = W.cnt[d * NSP].chunk0;
            const unsigned own = (unsigned)s_bc[sp];
            unsigned long long *lb = W.lb + (size_t)t * NSP + sp;
            unsigned excl = 0;
            if (t > first) {
                st_release(lb, (epoch << 32) | own);
                int j = t - 1;
                long long spins = 0;
                while (j >= first) {
                    unsigned long long v = ld_acquire(W.lb + (size_t)j * NSP + sp);
                    if ((v >> 32) != epoch) {
                        if (++spins > SPIN_LIMIT) {
                            set_status(ctl, ST_TIMEOUT);
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    excl += (unsigned)(v & 0x7FFFFFFFull);
                    if (v & 0x80000000ull) break;
                    --j;
                }
            }
            st_release(lb, (epoch << 32) | 0x80000000ull | (unsigned long long)(excl + own));
            s_bx[sp] = (int)excl;
            const int last = W.cnt[d * NSP + 2].chunk0 + W.cnt[d * NSP + 2].nchunk - 1;
            if (t == last) {
                Counts *cs = W.cnt + d * NSP + sp;
                const long long nn = (long long)cs->n_snap + excl + own;
                cs->n = (int)(nn < Dd.cap[sp] ? nn : Dd.cap[sp]);
            }
        }
        __syncthreads();
        for (int r = tid; r < nb; r += PUSH_THREADS) {
            const int sp = bTag[r] & 3;
            const long long dst = (long long)W.cnt[d * NSP + sp].n_snap + s_bx[sp] + bRank[r];
            if (dst >= Dd.cap[sp]) {
                set_status(ctl, ST_CAPACITY);
                continue;
            }
            const int g = Dd.pbase[sp] + (int)dst;
            cellA[g] = bCell[r];
            offA[g] = bOff[r];
            vxA[g] = bVx[r];
            vyA[g] = bVy[r];
            vzA[g] = bVz[r];
            deposit_global(accG + (size_t)sp * W.total_nodes + Dd.gbase, bCell[r], bOff[r], 1);
        }
        __syncthreads();
    }
    if (ds >= 0) flush(ds);
}

template <typename Real>
static size_t push_smem_bytes(int Nmax, int eedf_max, int fm_max)
{
    using Acc = typename AccT<Real>::T;
    size_t b = sizeof(Acc) * (Nmax + 2) + sizeof(Real) * (Nmax + 2);
    b += 4 * sizeof(Real) * BIRTH_CAP + 3 * sizeof(int) * BIRTH_CAP;
    b += sizeof(unsigned) * (eedf_max + fm_max);
    return (b + 15) & ~size_t(15);
}

cudaError_t push_configure(bool fp64, LaunchCfg &L, int num_sms)
{
    cudaError_t e;
    int per_sm = 1;
    if (fp64) {
        L.push_smem = push_smem_bytes<double>(L.maxN, 0, 0);
        L.push_smem_diag = push_smem_bytes<double>(L.maxN, L.eedf_max, L.fm_max);
        e = cudaFuncSetAttribute(k_push<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L.push_smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_push<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L.push_smem_diag);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<double, false>, PUSH_THREADS,
                                                          L.push_smem);
    } else {
        L.push_smem = push_smem_bytes<float>(L.maxN, 0, 0);
        L.push_smem_diag = push_smem_bytes<float>(L.maxN, L.eedf_max, L.fm_max);
        e = cudaFuncSetAttribute(k_push<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L.push_smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_push<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L.push_smem_diag);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<float, false>, PUSH_THREADS,
                                                          L.push_smem);
    }
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    L.push_blocks = num_sms * per_sm;
    return cudaSuccess;
}

cudaError_t launch_push(bool fp64, bool diag, const WsPtrs &W, const void *pools, int par,
                        const LaunchCfg &L, cudaStream_t st)
{
    const int em = diag ? L.eedf_max : 0, fm = diag ? L.fm_max : 0;
    const size_t sm = diag ? L.push_smem_diag : L.push_smem;
    if (fp64) {
        const Pools<double> &P = *static_cast<const Pools<double> *>(pools);
        if (diag)
            k_push<double, true><<<L.push_blocks, PUSH_THREADS, sm, st>>>(W, P, par, L.maxN, em, fm);
        else
            k_push<double, false><<<L.push_blocks, PUSH_THREADS, sm, st>>>(W, P, par, L.maxN, em, fm);
    } else {
        const Pools<float> &P = *static_cast<const Pools<float> *>(pools);
        if (diag)
            k_push<float, true><<<L.push_blocks, PUSH_THREADS, sm, st>>>(W, P, par, L.maxN, em, fm);
        else
            k_push<float, false><<<L.push_blocks, PUSH_THREADS, sm, st>>>(W, P, par, L.maxN, em, fm);
    }
    return cudaGetLastError();
}

} // namespace o2
