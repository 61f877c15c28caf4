// o2pic_push.cu -- the fused per-step particle kernel of libo2pic.
//
// One launch advances every live superparticle of every discharge by one time
// step (paper Sec. II (i) and Sec. III):
//   phase A, four consecutive slots per thread: gather E at x^n (linear
//   interpolation from a shared-memory copy of the node field) -> leapfrog
//   v^{n+1/2}, x^{n+1} -> absorption at x < 0 or x >= L -> null-collision
//   test against nu_max (one Philox4x32-10 block serves the four slots) ->
//   linear charge assignment of x^{n+1} into a per-block shared-memory grid
//   (warp aggregated, exact fixed point in the FP32 path) -> candidates
//   queued in shared memory;
//   phase B, one queued candidate per thread (no divergence across the
//   collision code): a gas molecule from the Maxwellian at T, the channel
//   walk over sum_j n_j sigma_j(E) u and the kinematics of the chosen
//   reaction; a particle that dies leaves the shared grid again; births are
//   staged per 1024-slot tile and appended in parent order by k_births.
//   The shared grid is flushed to the global accumulators with one atomic
//   per touched node.
//
// Particles are SoA with the position as (int32 cell, offset in [0,1)) and
// velocities in cells per step.  Slots are processed in tiles of 1024
// (256 threads x 4 consecutive slots, 16-byte vector loads); a persistent grid
// takes TILES_PER_TICKET tiles at a time from an atomic ticket.  No block ever
// waits for another.
#include <cstdio>

#include "o2pic_launch.h"

namespace o2 {

// three 256-thread blocks per SM in the FP32 path (the rare collision path
// may spill a little), two in the FP64 path
// tiles ahead of the current one whose particle data a push block asks the
// L2 cache to fetch (a bulk prefetch issued by one thread; 0 = none)
#ifndef O2_PUSH_L2_AHEAD
#define O2_PUSH_L2_AHEAD 2
#endif


template <typename Real> struct AccT;
template <> struct AccT<float> { using T = unsigned long long; };
template <> struct AccT<double> { using T = double; };

template <typename Real> struct GasTab;
template <> struct GasTab<float> {
    static constexpr int VEC = 4;
    static __device__ __forceinline__ const float *ptr(const WsPtrs &W) { return W.gtabf; }
    static __device__ __forceinline__ const float *bound(const WsPtrs &W) { return W.gpmf; }
    static __device__ __forceinline__ void load(const float *p, float v[4])
    {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <> struct GasTab<double> {
    static constexpr int VEC = 2;
    static __device__ __forceinline__ const double *ptr(const WsPtrs &W) { return W.gtab; }
    static __device__ __forceinline__ const double *bound(const WsPtrs &W) { return W.gpm; }
    static __device__ __forceinline__ void load(const double *p, double v[2])
    {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
        v[0] = t.x; v[1] = t.y;
    }
};

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

// the largest value below 1 (an offset that rounded up to 1 is held there)
template <typename Real> __device__ __forceinline__ Real below_one();
template <> __device__ __forceinline__ float below_one<float>() { return 0x1.fffffep-1f; }
template <> __device__ __forceinline__ double below_one<double>() { return 0x1.fffffffffffffp-1; }

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
    Real t = (log(E) - pick<Real>(T.lnE0, T.lnE0_f)) * pick<Real>(T.inv_dlog, T.inv_dlog_f);
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
    if (E < pick<Real>(T.th, T.th_f)) return Real(0);
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
struct BirthRec {
    int c;
    int tag;    // (slot in the sub-tile << 1 | product) << 2 | species
    Real off, vx, vy, vz;
};

// Births of one candidate go straight to its sub-tile's records, in any
// order; the tag restores parent order when they are appended.
template <typename Real>
struct BirthSink {
    BirthRec<Real> *rec;  // the sub-tile's birth_cap records
    int *n;               // the sub-tile's record count
    Ctl *ctl;
    int cap;
};

// ask the L2 cache to fetch [p, p + bytes) (16-byte aligned, a multiple of
// 16 bytes); no completion to wait for
__device__ __forceinline__ void l2_prefetch(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename Real>
__device__ __forceinline__ void stage_birth(const BirthSink<Real> &B, int tag, int sp, int c, Real off,
                                            const Real v[3])
{
    const int pos = atomicAdd(B.n, 1);
    if (pos >= B.cap) {
        set_status(B.ctl, ST_BIRTHBUF);
        return;
    }
    BirthRec<Real> &r = B.rec[pos];
    r.c = c;
    r.tag = (tag << 2) | sp;
    r.off = off;
    r.vx = v[0];
    r.vy = v[1];
    r.vz = v[2];
}

// Energy bin of an electron's lab energy K [eV] for the collision-frequency
// bound: with K = m 2^e, m in [1, 2), bin 4 (e + 6) + floor(4 (m - 1)) (the
// exponent and the top two mantissa bits), clamped to [0, nb - 1].  K is a
// sum of squares times a positive factor: for K >= 0 the exponent and the
// top two mantissa bits are the bits above the lower 21 (FP32), and +0 falls
// below bin 0.  (FP64: K <= 0 or NaN gives bin 0.)
__device__ __forceinline__ int energy_bin(float K, int nb)
{
    const int b = (int)(__float_as_uint(K) >> 21) - 4 * (127 + NUBIN_LOG2_E0);
    return min(max(b, 0), nb - 1);
}
__device__ __forceinline__ int energy_bin(double K, int nb)
{
    if (!(K > 0.0)) return 0;
    const unsigned long long u = (unsigned long long)__double_as_longlong(K);
    const int b = 4 * ((int)((u >> 52) & 0x7FFull) - 1023 - NUBIN_LOG2_E0) + (int)((u >> 50) & 3ull);
    return b < 0 ? 0 : (b > nb - 1 ? nb - 1 : b);
}

// One gas-target candidate (null-collision method).  Returns false if the
// particle died.  v is updated in place; products are staged.  The cell and
// offset are read from cP, offP (into c, off) only when the collision has
// products or kills the particle.
struct Outcome {
    bool alive;     // the particle survives
    bool viol;      // sum_j n_j sigma_j u exceeded the bound
    int reaction;   // reaction number, -1 for a null event
};

// Products of one gas event: species, product index (the tag's product
// bit) and velocity
template <typename Real>
struct GasProducts {
    int n;
    int sp[2], prod[2];
    Real v[2][3];
};

// Kinematics of gas channel ch for a particle of species s with velocity v
// that meets a gas molecule of velocity V at centre-of-mass energy E; nd is
// an isotropic direction, nd2 a second one used by (18).  Returns whether
// the particle lives on (with velocity vo) and its products.  One centre-of-
// mass scattering serves every channel that scatters: elastic (4), (5),
// isotropic (6) with no loss, (7)-(12) and (18) with the loss of Eq. 5; its
// result is unused by (15)-(17) and resonant (6).
template <typename Real>
__device__ __forceinline__ bool gas_event(const WsPtrs &W, const Disc &Dd, const SpeciesC &S, const GasChan &ch,
                                          const Real v[3], const Real V[3], Real E, const Real nd[3],
                                          const Real nd2[3], Real vo[3], GasProducts<Real> &pr)
{
    const int r = ch.reaction;
    const Real mf = pick<Real>(S.mfrac, S.mfrac_f), Mf = pick<Real>(S.Mfrac, S.Mfrac_f);
    const bool elastic = r <= 6;
    const bool dies = r >= 15 && r <= 17;
    Real Vo[3];
    cm_scatter<Real>(mf, Mf, v, V, elastic ? Real(0) : pick<Real>(ch.dloss, ch.dloss_f), nd, vo, Vo);
    const bool swap = r == 6 && !Dd.cx_iso;  // resonant exchange: the ion takes the gas velocity
#pragma unroll
    for (int q = 0; q < 3; ++q) vo[q] = swap ? V[q] : vo[q];
    pr.n = 0;
    if (r == 18) {
        // ionisation: the O2 splits into O2+ and a second electron with the
        // post-collision O2 velocity, then the two electrons collide
        // elastically (isotropic in their centre of mass)
        Real e2[3] = {Vo[0], Vo[1], Vo[2]};
        ee_elastic<Real>(vo, e2, nd2);
        pr.n = 2;
        pr.sp[0] = 0;
        pr.prod[0] = 0;
        pr.sp[1] = 2;
        pr.prod[1] = 1;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            pr.v[0][q] = e2[q];
            pr.v[1][q] = Vo[q];
        }
    }
    if (!dies) return true;
    // (15) attachment: O- with the CM velocity plus half the relative
    // energy above threshold shared back to back with O; (16) detachment:
    // electron with a tenth of the O- energy, isotropic; (17) associative
    // detachment: electron with the CM energy about the CM velocity
    Real w;
    if (r == 16) {
        w = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) * pick<Real>(Dd.f16, Dd.f16_f);
    } else {
        Real arg;
        if (r == 15) {
            const TableDesc &Tc = W.tables[ch.table];
            const Real Ea = E - pick<Real>(Tc.th, Tc.th_f);
            arg = (Ea > Real(0) ? Ea : Real(0)) * pick<Real>(Dd.f15, Dd.f15_f);
        } else {
            arg = E * pick<Real>(Dd.f17, Dd.f17_f);
        }
        w = sqrt(arg);
    }
    const Real A = r == 16 ? Real(0) : Real(1);
    pr.n = 1;
    pr.sp[0] = r == 15 ? 1 : 0;
    pr.prod[0] = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) pr.v[0][q] = A * (mf * v[q] + Mf * V[q]) + w * nd[q];
    return false;
}

template <typename Real>
__device__ __forceinline__ Outcome gas_collide(const WsPtrs &W, const Disc &Dd, int s, unsigned idx,
                                            unsigned long long step, Real numax_n, Real &vx, Real &vy,
                                            Real &vz, const int *cP, const Real *offP, int &c, Real &off,
                                            int tag, const BirthSink<Real> &B)
{
    const SpeciesC &S = Dd.sp[s];
    const Real *lutE = Lut<Real>::E(W);
    const Real *lutS = Lut<Real>::S(W);
    uint4 a = rng_block(Dd.seed, Dd.discharge, s, 1, 0, 0, step, idx);
    uint4 b = rng_block(Dd.seed, Dd.discharge, s, 1, 0, 1, step, idx);
    Real n0, n1, n2, n3;
    box_muller<Real>(a.x, a.y, n0, n1);
    box_muller<Real>(a.z, a.w, n2, n3);
    const Real vg = pick<Real>(S.vgas_n, S.vgas_n_f);
    Real V[3] = {vg * n0, vg * n1, vg * n2};
    Real v[3] = {vx, vy, vz};
    Real g0 = v[0] - V[0], g1 = v[1] - V[1], g2 = v[2] - V[2];
    Real u2 = g0 * g0 + g1 * g1 + g2 * g2;
    Real u = sqrt(u2);
    Real E = pick<Real>(S.Ek, S.Ek_f) * u2;
    Real target = unif<Real>(b.x) * numax_n;
    const TableDesc &T0 = W.tables[S.table_lo];
    XsPoint<Real> pt = xs_locate<Real>(T0, lutE, E);
    // node-major table of n_j dx sigma_j(E_k): the rows k and k+1 of every
    // channel come in a few 16-byte loads
    const Real *row = GasTab<Real>::ptr(W) + S.gtab_off;
    const int ld = S.gtab_ld;
    const Real *ra = row + (size_t)pt.k * ld;
    const Real *rb = ra + ld;
    Real cum = Real(0);
    int chosen = -1;
    // channel walk with selects only: the lanes of a warp stay together
    for (int j0 = 0; j0 < S.nch; j0 += GasTab<Real>::VEC) {
        Real a[GasTab<Real>::VEC], b[GasTab<Real>::VEC];
        GasTab<Real>::load(ra + j0, a);
        GasTab<Real>::load(rb + j0, b);
#pragma unroll
        for (int q = 0; q < GasTab<Real>::VEC; ++q) {
            const int j = j0 + q;
            if (j >= S.nch) break;  // uniform: one species per warp
            // below the grid f = 0 gives a exactly; above it, the last node
            Real v = pt.region == 2 ? b[q] : a[q] + pt.f * (b[q] - a[q]);
            v = E < pick<Real>(S.ch[j].th, S.ch[j].th_f) ? Real(0) : v;
            cum += v * u;
            chosen = (chosen < 0 && target < cum) ? j : chosen;
        }
    }
    const bool viol = cum > numax_n;
    if (chosen < 0) return Outcome{true, viol, -1};  // null event
    const GasChan &ch = S.ch[chosen];
    const int r = ch.reaction;
    Real nd[3], nd2[3] = {Real(0), Real(0), Real(1)};
    iso_dir<Real>(unif<Real>(b.y), unif<Real>(b.z), nd);
    if (r == 18) {
        uint4 e = rng_block(Dd.seed, Dd.discharge, s, 1, 0, 2, step, idx);
        iso_dir<Real>(unif<Real>(e.x), unif<Real>(e.y), nd2);
    }
    GasProducts<Real> pr;
    Real vo[3];
    const bool alive = gas_event<Real>(W, Dd, S, ch, v, V, E, nd, nd2, vo, pr);
    // the position is needed only by products and by a dying particle
    if (pr.n > 0 || !alive) {
        c = *cP;
        off = *offP;
    }
    for (int q = 0; q < pr.n; ++q) stage_birth<Real>(B, tag | pr.prod[q], pr.sp[q], c, off, pr.v[q]);
    if (alive) {
        vx = vo[0]; vy = vo[1]; vz = vo[2];
    }
    return Outcome{alive, viol, r};
}

template <typename Acc> __device__ __forceinline__ void acc_add(Acc *a, Acc v);
template <> __device__ __forceinline__ void acc_add(unsigned long long *a, unsigned long long v)
{
    atomicAdd(a, v);
}
template <> __device__ __forceinline__ void acc_add(double *a, double v) { atomicAdd(a, v); }

// Split 64-bit shared sums of the FP32 path: the 8 bytes hold two signed
// 32-bit sums, of the low SPLIT_BITS bits of each added weight (word 0) and
// of the rest (word 1); the value is word1 * 2^SPLIT_BITS + word0.  Adds are
// plain 32-bit atomics whose result is not needed (no carry), and both sums
// stay exact while a block adds at most FLUSH_TICKETS tickets of weights
// before it flushes (each particle's weight is at most 2^FIX_BITS, so word 1
// grows by at most 2^(FIX_BITS - SPLIT_BITS) per particle and word 0 by less
// than 2^SPLIT_BITS per add).
constexpr int SPLIT_BITS = 12;
constexpr int FLUSH_TICKETS = 256 / TILES_PER_TICKET;  // 256 tiles of weights at most
static_assert((long long)FLUSH_TICKETS * TILES_PER_TICKET * CHUNK * (1LL << (FIX_BITS - SPLIT_BITS)) < (1LL << 31),
              "split sums must stay within int32");
__device__ __forceinline__ void split_add(unsigned long long *node, unsigned v)
{
    unsigned *w = reinterpret_cast<unsigned *>(node);  // w[0] low part, w[1] high part
    atomicAdd(&w[0], v & ((1u << SPLIT_BITS) - 1u));
    atomicAdd(&w[1], v >> SPLIT_BITS);
}
__host__ __device__ __forceinline__ unsigned long long split_value(unsigned long long node)
{
    const long long lo = (int)(unsigned)(node & 0xFFFFFFFFull);
    const long long hi = (int)(unsigned)(node >> 32);
    return (unsigned long long)(hi * (1LL << SPLIT_BITS) + lo);
}

// The FP64 path's shared grid holds exact 64-bit integer sums of the
// weights in units of 2^-FIX_BITS_64 (a particle's two weights add up to
// exactly 2^FIX_BITS_64); they become doubles once per node and flush.  A
// block adds at most FLUSH_TICKETS tickets of weights before a flush, far
// below the 2^63 / 2^FIX_BITS_64 particles a node could hold.  (Shared-memory
// double atomics took nine tenths of the FP64 push.)
constexpr int FIX_BITS_64 = 40;
static_assert((long long)FLUSH_TICKETS * TILES_PER_TICKET * CHUNK < (1LL << (63 - FIX_BITS_64)),
              "FP64 shared sums must stay within int64");

// the block's sum of a node in the global accumulators' type
template <typename Real> __device__ __forceinline__ typename AccT<Real>::T sacc_value(unsigned long long node);
template <> __device__ __forceinline__ unsigned long long sacc_value<float>(unsigned long long node)
{
    return split_value(node);
}
template <> __device__ __forceinline__ double sacc_value<double>(unsigned long long node)
{
    return (double)(long long)node * (1.0 / (double)(1ull << FIX_BITS_64));
}

// a node's sum in the global accumulators' type from the block's shared sums
template <typename Real>
__device__ __forceinline__ typename AccT<Real>::T sacc_node(const unsigned long long *sAcc, const unsigned *sCnt, int i);
template <>
__device__ __forceinline__ unsigned long long sacc_node<float>(const unsigned long long *sAcc, const unsigned *sCnt,
                                                               int i)
{
    const unsigned long long lw = i > 0 ? split_value(sAcc[i - 1]) : 0ull;
    return ((unsigned long long)sCnt[i] << FIX_BITS) - split_value(sAcc[i]) + lw;
}
template <>
__device__ __forceinline__ double sacc_node<double>(const unsigned long long *sAcc, const unsigned *, int i)
{
    return sacc_value<double>(sAcc[i]);
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

// Charge of the four slots of a thread into the block's shared sums.  The
// FP32 sums are kept per CELL: the particles that land in it (sCnt, one
// 32-bit add) and the sum of their upper CIC weights w1 = rn(offset
// 2^FIX_BITS) (sAcc, split words); node i is then
// count_i 2^FIX_BITS - W1_i + W1_(i-1), the same integer as the sum of the
// particles' two node weights, with three shared atomics per particle
// instead of four.  When the whole warp's slots sit in one cell (sorted,
// slow particles) the weights are summed over the warp and one lane adds
// them; otherwise every lane adds its own (its four summed first when they
// share a cell; 4 * 32 * 2^FIX_BITS < 2^32).  No lane matching: it runs on a
// narrow pipe.
__device__ __forceinline__ void deposit4(unsigned long long *sAcc, unsigned *sCnt, const int dep[4],
                                         const float off[4])
{
    unsigned w1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w1[k] = dep[k] >= 0 ? __float2uint_rn(off[k] * (float)(1 << FIX_BITS)) : 0u;
    const int lane = threadIdx.x & 31;
    const bool same = dep[0] >= 0 && dep[1] == dep[0] && dep[2] == dep[0] && dep[3] == dep[0];
    const unsigned a = w1[0] + w1[1] + w1[2] + w1[3];
    const int c0 = __shfl_sync(0xffffffffu, dep[0], 0);
    if (__all_sync(0xffffffffu, same && dep[0] == c0)) {
        const unsigned sa = __reduce_add_sync(0xffffffffu, a);
        if (lane == 0) {
            atomicAdd(&sCnt[c0], 128u);
            split_add(&sAcc[c0], sa);
        }
        return;
    }
    if (same) {
        atomicAdd(&sCnt[dep[0]], 4u);
        split_add(&sAcc[dep[0]], a);
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // an empty slot adds nothing to cell 0
        const int ck = dep[k] >= 0 ? dep[k] : 0;
        atomicAdd(&sCnt[ck], dep[k] >= 0 ? 1u : 0u);
        split_add(&sAcc[ck], w1[k]);
    }
}

// The push that also samples the diagnostics keeps its FP32 sums per NODE
// (both CIC weights of a particle, split words, four shared atomics per
// particle): its shared memory holds the histograms, and per-cell counts on
// top of them would leave room for fewer blocks per SM.
__device__ __forceinline__ void deposit4_nodes(unsigned long long *sAcc, const int dep[4], const float off[4])
{
    unsigned w0[4], w1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        w1[k] = dep[k] >= 0 ? __float2uint_rn(off[k] * (float)(1 << FIX_BITS)) : 0u;
        w0[k] = dep[k] >= 0 ? (1u << FIX_BITS) - w1[k] : 0u;
    }
    const int lane = threadIdx.x & 31;
    const bool same = dep[0] >= 0 && dep[1] == dep[0] && dep[2] == dep[0] && dep[3] == dep[0];
    const unsigned a = w0[0] + w0[1] + w0[2] + w0[3];
    const unsigned b = w1[0] + w1[1] + w1[2] + w1[3];
    const int c0 = __shfl_sync(0xffffffffu, dep[0], 0);
    if (__all_sync(0xffffffffu, same && dep[0] == c0)) {
        const unsigned sa = __reduce_add_sync(0xffffffffu, a);
        const unsigned sb = __reduce_add_sync(0xffffffffu, b);
        if (lane == 0) {
            split_add(&sAcc[c0], sa);
            split_add(&sAcc[c0 + 1], sb);
        }
        return;
    }
    if (same) {
        split_add(&sAcc[dep[0]], a);
        split_add(&sAcc[dep[0] + 1], b);
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        // an empty slot adds zero weights to node 0
        const int ck = dep[k] >= 0 ? dep[k] : 0;
        split_add(&sAcc[ck], w0[k]);
        split_add(&sAcc[ck + 1], w1[k]);
    }
}
__device__ __forceinline__ void deposit4_nodes(unsigned long long *sAcc, const int dep[4], const double off[4])
{
    constexpr double SC = (double)(1ull << FIX_BITS_64);
    unsigned long long w0[4], w1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        w1[k] = dep[k] >= 0 ? (unsigned long long)__double2ll_rn(off[k] * SC) : 0ull;
        w0[k] = dep[k] >= 0 ? (1ull << FIX_BITS_64) - w1[k] : 0ull;
    }
    // as in the FP32 path: a warp whose 128 slots sit in one cell adds its
    // sums once, a lane whose four slots share a cell adds them once
    const int lane = threadIdx.x & 31;
    const bool same = dep[0] >= 0 && dep[1] == dep[0] && dep[2] == dep[0] && dep[3] == dep[0];
    unsigned long long a = w0[0] + w0[1] + w0[2] + w0[3];
    unsigned long long b = w1[0] + w1[1] + w1[2] + w1[3];
    const int c0 = __shfl_sync(0xffffffffu, dep[0], 0);
    if (__all_sync(0xffffffffu, same && dep[0] == c0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            atomicAdd(&sAcc[c0], a);
            atomicAdd(&sAcc[c0 + 1], b);
        }
        return;
    }
    if (same) {
        atomicAdd(&sAcc[dep[0]], a);
        atomicAdd(&sAcc[dep[0] + 1], b);
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (dep[k] >= 0) {
            atomicAdd(&sAcc[dep[k]], w0[k]);
            atomicAdd(&sAcc[dep[k] + 1], w1[k]);
        }
    }
}

// the species of (discharge, species) index ds has an energy-binned bound
__device__ __forceinline__ bool Dd_binned(const WsPtrs &W, int ds)
{
    return W.disc[ds / NSP].sp[ds % NSP].nbins > 0;
}

// Push arithmetic of a lane's four slots: E at the particle by linear
// interpolation, v + (q/m) E dt, offset + v dt / dx.  FP32: two slots per
// packed instruction (the same roundings as the scalar fused multiply-adds).
template <typename Real>
__device__ __forceinline__ void push_arith(const Real *sE, const int c[4], const Real off[4], const Real vx[4],
                                           Real qm, Real ks, Real vn[4], Real on[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int cc = c[k] >= 0 ? c[k] : 0;
        const Real e0 = sE[cc], e1 = sE[cc + 1];
        const Real ep = e0 + off[k] * (e1 - e0);
        vn[k] = vx[k] + qm * ep;
        on[k] = off[k] + vn[k] * ks;
    }
}
template <>
__device__ __forceinline__ void push_arith<float>(const float *sE, const int c[4], const float off[4],
                                                  const float vx[4], float qm, float ks, float vn[4], float on[4])
{
    const float2 qm2 = make_float2(qm, qm), ks2 = make_float2(ks, ks);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int ca = c[2 * p] >= 0 ? c[2 * p] : 0, cb = c[2 * p + 1] >= 0 ? c[2 * p + 1] : 0;
        const float2 e0 = make_float2(sE[ca], sE[cb]);
        const float2 e1 = make_float2(sE[ca + 1], sE[cb + 1]);
        const float2 of = make_float2(off[2 * p], off[2 * p + 1]);
        const float2 v0 = make_float2(vx[2 * p], vx[2 * p + 1]);
        const float2 de = __fadd2_rn(e1, make_float2(-e0.x, -e0.y));
        const float2 ep = __ffma2_rn(of, de, e0);
        const float2 v = __ffma2_rn(qm2, ep, v0);
        const float2 o = __ffma2_rn(v, ks2, of);
        vn[2 * p] = v.x;
        vn[2 * p + 1] = v.y;
        on[2 * p] = o.x;
        on[2 * p + 1] = o.y;
    }
}
// lab kinetic energy factor ke (v^2 + vy^2 + vz^2) of four slots
template <typename Real>
__device__ __forceinline__ void energy2(Real ke, const Real v[4], const Real vy[4], const Real vz[4], Real K[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) K[k] = ke * (v[k] * v[k] + vy[k] * vy[k] + vz[k] * vz[k]);
}
template <>
__device__ __forceinline__ void energy2<float>(float ke, const float v[4], const float vy[4], const float vz[4],
                                               float K[4])
{
    const float2 ke2 = make_float2(ke, ke);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float2 a = make_float2(v[2 * p], v[2 * p + 1]);
        const float2 y = make_float2(vy[2 * p], vy[2 * p + 1]);
        const float2 z = make_float2(vz[2 * p], vz[2 * p + 1]);
        float2 t = __fmul2_rn(a, a);
        t = __ffma2_rn(y, y, t);
        t = __ffma2_rn(z, z, t);
        t = __fmul2_rn(ke2, t);
        K[2 * p] = t.x;
        K[2 * p + 1] = t.y;
    }
}

// Launch shape of the push: NT threads per block, SPT slots per thread.  A
// warp takes SPT/4 consecutive sub-tiles of 128 slots per pass and lane l the
// four consecutive slots 4l .. 4l+3 of each (16-byte vectors, one Philox
// block); a block's pass covers NT SPT / 128 sub-tiles.  MINB is the blocks
// per SM the register allocation is sized for.
template <int NT, int SPT, int MINB>
struct PushShape {
    static constexpr int threads = NT;
    static constexpr int spt = SPT;
    static constexpr int minb = MINB;
    static constexpr int nw = NT / 32;
    static constexpr int groups = SPT / 4;                 // sub-tiles per warp and pass
    static constexpr int qcap = 32 + 32 * SPT;             // candidate queue: < 32 left + one pass
    static_assert(SPT % 4 == 0 && NT % 32 == 0, "shape");
    static_assert((TILES_PER_TICKET * SUBTILES) % (nw * groups) == 0, "a ticket holds whole passes");
};

template <typename Real, bool DIAG, typename SH>
__global__ void __launch_bounds__(SH::threads, SH::minb)
k_push(WsPtrs W, Pools<Real> P, int par, int Nmax, int eedf_max, int fm_max)
{
    pdl_wait();
    using Acc = typename AccT<Real>::T;
    constexpr int PUSH_THREADS = SH::threads, NW = SH::nw, G = SH::groups, QCAP = SH::qcap;
    // FP32 without diagnostics: per-cell sums (counts + upper weights)
    constexpr bool CELLS = sizeof(Real) == 4 && !DIAG;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *sAcc = reinterpret_cast<unsigned long long *>(smem);  // integer sums (both paths)
    Real *sE = reinterpret_cast<Real *>(sAcc + (Nmax + 2));
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // per-warp list of collision candidates (slot, energy bin) before it is
    // written out, and the histograms
    int *qIdx = reinterpret_cast<int *>(sE + (Nmax + 2)) + w * QCAP;
    unsigned *sEedf = reinterpret_cast<unsigned *>(sE + (Nmax + 2)) + NW * QCAP;
    unsigned *sFm = sEedf + eedf_max;
    unsigned char *qBin = reinterpret_cast<unsigned char *>(sFm + fm_max) + w * QCAP;
    // FP32: particles per cell of the block's sums, after the queues' bins
    unsigned *sCnt = reinterpret_cast<unsigned *>(
        (reinterpret_cast<size_t>(reinterpret_cast<unsigned char *>(sFm + fm_max) + NW * QCAP) + 15) & ~size_t(15));

    __shared__ int s_ticket[2];
    __shared__ unsigned s_cnt[C_NCOUNT];
    __shared__ unsigned s_btn[NUBIN_MAX];  // electron bounds per energy bin: thresholds

    Ctl *ctl = W.ctl;
    const int cur = ctl->cur;
    const unsigned long long step = ctl->step[par];
    const int total = ctl->total_chunks;
    const int nds = W.D * NSP;
    int *cellA = P.cell[cur];
    Real *offA = P.off[cur], *vxA = P.vx[cur], *vyA = P.vy[cur], *vzA = P.vz[cur];
    Acc *accG = acc_global<Real>(W);
    const unsigned lt_mask = (1u << lane) - 1u;

    int ds = -1, d = -1, run_tk = 0;
    for (int q = tid; q < C_NCOUNT; q += PUSH_THREADS) s_cnt[q] = 0;
    auto flush = [&](int fds) {
        const int fd = fds / NSP, fs = fds % NSP;
        const Disc &Dd = W.disc[fd];
        __syncthreads();
        Acc *g = accG + (size_t)fs * W.total_nodes + Dd.gbase;
        for (int i = tid; i <= Dd.N; i += PUSH_THREADS) {
            const Acc v = CELLS ? sacc_node<Real>(sAcc, sCnt, i) : sacc_value<Real>(sAcc[i]);
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

    // ---- the warp's candidates go to the step's list (one reservation per
    // batch); the collision kernel takes them from there
    int qn = 0;  // warp-uniform
    auto list_out = [&]() {
        int base = 0;
        if (lane == 0) {
            base = (int)atomicAdd(&ctl->cand_n, (unsigned)qn);
            atomicAdd(&s_cnt[C_CANDS], (unsigned)qn);
            if (Dd_binned(W, ds)) atomicAdd(&s_cnt[C_BCANDS], (unsigned)qn);
            if ((long long)base + qn > W.cand_cap) set_status(ctl, ST_BIRTHBUF);
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        for (int q = lane; q < qn; q += 32) {
            const long long at = (long long)base + q;
            if (at < W.cand_cap) W.cand[at] = make_int2(qIdx[q], (ds << 8) | qBin[q]);
        }
        __syncwarp();
        qn = 0;
    };

    for (int it = 0;; ++it) {
        // two ticket buffers: a buffer is rewritten only after the barrier
        // that every reader of its previous value has passed
        if (tid == 0) s_ticket[it & 1] = (int)atomicAdd(&ctl->ticket, (unsigned)TILES_PER_TICKET);
        __syncthreads();
        const int tbeg = s_ticket[it & 1];
        if (tbeg >= total) break;
        // tiles of one (discharge, species) start at a multiple of
        // TILES_PER_TICKET, so a ticket belongs to one (d, s) or to padding
        int nx = ds < 0 ? 0 : ds;
        while (nx < nds && !(tbeg >= W.cnt[nx].chunk0 && tbeg < W.cnt[nx].chunk0 + W.cnt[nx].nchunk)) ++nx;
        if (nx >= nds) continue;
        if (species_rests(W.disc[nx / NSP], nx % NSP, step)) {
            // a resting ion species: nothing to push; its sub-tiles record no births
            const int te = min(tbeg + TILES_PER_TICKET, W.cnt[nx].chunk0 + W.cnt[nx].nchunk);
            for (int q = tid; q < (te - tbeg) * SUBTILES; q += PUSH_THREADS)
                W.tile_cnt[((size_t)tbeg * SUBTILES + q) * NSP] = 0;
            continue;
        }
        // a new (d, s), or the block's integer sums at their bound: flush
        if (nx != ds || run_tk >= FLUSH_TICKETS) {
            if (qn > 0) list_out();
            if (ds >= 0) flush(ds);
            const int nd = nx / NSP;
            const Disc &Dn = W.disc[nd];
            if (nd != d) {
                const Real *Eg = reinterpret_cast<const Real *>(W.Ereal) + Dn.gbase;
                for (int i = tid; i <= Dn.N; i += PUSH_THREADS) sE[i] = Eg[i];
                d = nd;
            }
            for (int i = tid; i <= Dn.N + 1; i += PUSH_THREADS) {
                sAcc[i] = 0ull;
                if (CELLS) sCnt[i] = 0u;
            }
            {
                const SpeciesC &Sn = Dn.sp[nx % NSP];
                for (int b = tid; b < Sn.nbins; b += PUSH_THREADS) {
                    const NuBin &nb = W.nubin[Sn.bin_off + b];
                    s_btn[b] = nb.tnull;
                }
            }
            for (int q = tid; q < C_NCOUNT; q += PUSH_THREADS) s_cnt[q] = 0;
            if (DIAG) {
                for (int i = tid; i < eedf_max; i += PUSH_THREADS) sEedf[i] = 0;
                for (int i = tid; i < fm_max; i += PUSH_THREADS) sFm[i] = 0;
            }
            ds = nx;
            run_tk = 0;
            __syncthreads();
        }
        ++run_tk;
        const int s = ds % NSP;
        const Disc &Dd = W.disc[d];
        const SpeciesC &S = Dd.sp[s];
        const Counts &C = W.cnt[ds];
        const int N = Dd.N;
        const int pb = Dd.pbase[s];
        const int end = pb + C.n_snap;
        const int tend = min(tbeg + TILES_PER_TICKET, C.chunk0 + C.nchunk);
        // a sub-cycled ion species moves over ks steps per push
        const Real ks = Real(s > 0 ? Dd.ion_sub : 1);
        const Real qm = pick<Real>(S.qm, S.qm_f) * ks;
        const unsigned tnull = S.tnull;
        const int nbins = S.nbins;
        const bool binned = nbins > 0;  // electrons: bound per lab-energy bin
        const Real ke = pick<Real>(S.ke_eV, S.ke_eV_f);
        const float rN = 1.0f / (float)N;  // the diagnostics' x bins
        // the ticket's sub-tiles in rows of NW G: warp w takes sub-tiles
        // w G .. w G + G - 1 of every row
        constexpr int ROW = NW * G;
        const int st_beg = tbeg * SUBTILES, st_end = tend * SUBTILES;
        // the warp's first slot in the ticket
        const int wbase0 = pb + (tbeg - C.chunk0) * CHUNK + w * G * SUBTILE;
        unsigned tslots = 0, tlive = 0;  // the ticket's slot counts of this thread
        for (int r0 = st_beg; r0 < st_end; r0 += ROW) {
            if (O2_PUSH_L2_AHEAD > 0 && tid == 0) {
                // the row O2_PUSH_L2_AHEAD ahead in this ticket (on the first
                // row also those between): cell, offset and vx into L2
                const int ra = (r0 == st_beg) ? r0 + ROW : r0 + O2_PUSH_L2_AHEAD * ROW;
                const int rb = (r0 == st_beg) ? min(r0 + O2_PUSH_L2_AHEAD * ROW, st_end - ROW) : ra;
                for (int rp = ra; rp <= rb && rp < st_end; rp += ROW) {
                    const size_t sl = (size_t)pb + (size_t)(rp - C.chunk0 * SUBTILES) * SUBTILE;
                    const unsigned n = (unsigned)min(ROW, st_end - rp) * SUBTILE;
                    l2_prefetch(cellA + sl, n * sizeof(int));
                    l2_prefetch(offA + sl, n * sizeof(Real));
                    l2_prefetch(vxA + sl, n * sizeof(Real));
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
            const int sub = r0 + w * G + g;
            // a row of at most one tile fits the ticket's whole tiles; a
            // longer one can overhang its tail
            if (ROW > SUBTILES && sub >= st_end) break;
            const int i0 = wbase0 + (r0 - st_beg) * SUBTILE + g * SUBTILE + 4 * lane;
            if (lane == 0) W.tile_cnt[(size_t)sub * NSP] = 0;  // births recorded by the collision kernel

            // ---- phase A: push, absorb, null test, deposit, candidate queue
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
            Real vyl[4], vzl[4];  // binned species only: the lab energy needs vy, vz
            if (binned) {
                if (full) {
                    ld4(vyA + i0, vyl);
                    ld4(vzA + i0, vzl);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const bool in = i0 + k < end;
                        vyl[k] = in ? vyA[i0 + k] : Real(0);
                        vzl[k] = in ? vzA[i0 + k] : Real(0);
                    }
                }
            }
            uint4 w4 = make_uint4(0, 0, 0, 0);
            if (c[0] >= 0 || c[1] >= 0 || c[2] >= 0 || c[3] >= 0)
                w4 = rng_block(Dd.seed, Dd.discharge, s, 0, 0, 0, step, (unsigned)((i0 - pb) >> 2));
            const unsigned wk[4] = {w4.x, w4.y, w4.z, w4.w};
            // each slot is pushed without branches; absorptions are noted in
            // a mask and handled after the four slots
            unsigned nslots = 0, nlive = 0, outm = 0, wallm = 0;
            bool cchg = false;  // a cell index of the lane's slots changed
            bool nonfin = false;
            unsigned candm = 0u, bins = 0u;
            int dep[4];
            // the field at the particle, the new velocity and position (the
            // FP32 path takes two slots per packed instruction)
            Real vn[4], on[4], Kn[4];
            push_arith<Real>(sE, c, off, vx, qm, ks, vn, on);
            if (binned) energy2<Real>(ke, vn, vyl, vzl, Kn);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int ck = c[k];
                const bool was = ck >= 0;
                nslots += ck >= -1 ? 1u : 0u;
                nlive += was ? 1u : 0u;
                const int cc = was ? ck : 0;
                const Real v = vn[k];
                Real o = on[k];
                const Real fl = floor(o);
                const bool bad = !(fl > Real(-2 * N - 4) && fl < Real(2 * N + 4));
                // a non-finite velocity or position is an error, not an absorption
                nonfin |= was && !isfinite(o);
                int cn = bad ? (v < Real(0) ? -1 : N) : cc + (int)fl;
                o -= fl;
                const bool wrap = o >= Real(1);
                o = wrap ? o - Real(1) : o;
                cn += wrap ? 1 : 0;
                const bool out = was && (cn < 0 || cn >= N);
                const bool live = was && !out;
                outm |= (out && isfinite(o)) ? 1u << k : 0u;
                wallm |= cn >= N ? 1u << k : 0u;
                vx[k] = was ? v : vx[k];
                off[k] = live ? o : off[k];
                const int cnew = was ? (out ? -1 : cn) : ck;
                cchg |= cnew != ck;
                c[k] = cnew;
                dep[k] = live ? cn : -1;
                int bin = 0;
                unsigned thr = tnull;
                if (binned) {
                    bin = energy_bin(Kn[k], nbins);
                    thr = s_btn[bin];
                }
                const bool cand = live && wk[k] < thr;
                candm |= cand ? 1u << k : 0u;
                bins |= (unsigned)bin << (8 * k);
            }
            // candidates are rare: one vote, and the queue only when a lane has one
            if (__any_sync(0xffffffffu, candm != 0u)) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const bool cand = (candm >> k) & 1u;
                    const unsigned m = __ballot_sync(0xffffffffu, cand);
                    if (cand) {
                        const int pos = qn + __popc(m & lt_mask);
                        qIdx[pos] = i0 + k;
                        qBin[pos] = (unsigned char)(bins >> (8 * k));
                    }
                    qn += __popc(m);
                }
            }
            if (nonfin) set_status(ctl, ST_NONFINITE);
            if (outm) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (!((outm >> k) & 1u)) continue;
                    const int wall = (wallm >> k) & 1u;
                    atomicAdd(&s_cnt[C_ABS + 2 * s + wall], 1u);
                    if (s == 2 && Dd.iedf_bins > 0) {
                        const Real v = vx[k], vy = vyA[i0 + k], vz = vzA[i0 + k];
                        const Real Ei = pick<Real>(S.ke_eV, S.ke_eV_f) * (v * v + vy * vy + vz * vz);
                        const Real bb = floor(Ei * pick<Real>(Dd.iedf_scale, Dd.iedf_scale_f));
                        if (bb >= Real(0) && bb < Real(Dd.iedf_bins))
                            atomicAdd(&W.iedf[Dd.iedf_base + wall * Dd.iedf_bins + (int)bb], 1u);
                    }
                }
            }
            if (DIAG) {
                // distributions after the free flight, before collisions
                if (s == 0 && Dd.eedf_bins > 0) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (dep[k] != N / 2) continue;
                        const Real v = vx[k], vy = vyA[i0 + k], vz = vzA[i0 + k];
                        const Real Ee = pick<Real>(S.ke_eV, S.ke_eV_f) * (v * v + vy * vy + vz * vz);
                        const Real bb = floor(Ee * pick<Real>(Dd.eedf_scale, Dd.eedf_scale_f));
                        if (bb >= Real(0) && bb < Real(Dd.eedf_bins)) atomicAdd(&sEedf[(int)bb], 1u);
                    }
                }
                if (s == 1 && Dd.fm_bins > 0) {
                    // cold, sorted O- of a warp fall into a few bins: the lanes
                    // of one bin add their count once (no 32-way conflicts)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int cn = dep[k];
                        int fb = -1;
                        if (cn >= 0) {
                            const Real v = vx[k];
                            Real Es = pick<Real>(S.ke_eV, S.ke_eV_f) * v * v;
                            if (v < Real(0)) Es = -Es;
                            const Real bb = floor((Es + pick<Real>(Dd.fm_emax, Dd.fm_emax_f)) *
                                                  pick<Real>(Dd.fm_scale, Dd.fm_scale_f));
                            if (bb >= Real(0) && bb < Real(Dd.fm_bins)) {
                                // x bin floor(cn X / N) without an integer division: an
                                // estimate through 1/N in FP32 (off by at most one, as
                                // cn X <= 2^26), then corrected
                                const int pr = cn * Dd.fm_xbins;
                                int xb = (int)((float)pr * rN);
                                xb += (xb + 1) * N <= pr ? 1 : 0;
                                xb -= xb * N > pr ? 1 : 0;
                                fb = xb * Dd.fm_bins + (int)bb;
                            }
                        }
                        const unsigned peers = __match_any_sync(0xffffffffu, fb);
                        if (fb >= 0 && lane == __ffs(peers) - 1) atomicAdd(&sFm[fb], (unsigned)__popc(peers));
                    }
                }
            }
            if constexpr (CELLS)
                deposit4(sAcc, sCnt, dep, off);
            else
                deposit4_nodes(sAcc, dep, off);
            tslots += nslots;
            tlive += nlive;
            if (full) {
                // an unchanged value is not written back: slow ions keep
                // their cells for many steps, and a lane of dead slots
                // changes nothing (its DRAM sectors then stay clean)
                if (cchg) st4(cellA + i0, c);
                if (nlive) {
                    st4(offA + i0, off);
                    st4(vxA + i0, vx);
                }
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
            }
            __syncwarp();
            if (qn >= 32) list_out();
        }
        {
            const unsigned ws = __reduce_add_sync(0xffffffffu, tslots);
            const unsigned wl = __reduce_add_sync(0xffffffffu, tlive);
            if (lane == 0) {
                if (ws) atomicAdd(&s_cnt[C_SLOTS], ws);
                if (ws && binned) atomicAdd(&s_cnt[C_BSLOTS], ws);
                if (wl) atomicAdd(&s_cnt[C_LIVE], wl);
            }
        }
    }
    if (qn > 0) list_out();
    if (ds >= 0) flush(ds);
}


// Collisions of the step's candidates (null-collision method, Sec. III
// kinematics): one thread per candidate, in list order; a dying particle's
// charge leaves the global grid, births go to its sub-tile's records.  A
// candidate's cell and offset are read only when its collision has products
// or kills it, and its velocity is written back only after an event (a
// null event changes nothing): each field is a scattered access.  Event
// counts are summed per block for the discharge of the block's first
// candidate (the list holds runs of one discharge), others go straight to
// the global counters.
#ifndef O2_COLLIDE_MIN_BLOCKS
#define O2_COLLIDE_MIN_BLOCKS 1
#endif
template <typename Real>
__global__ void __launch_bounds__(COLLIDE_THREADS, O2_COLLIDE_MIN_BLOCKS)
k_collide(WsPtrs W, Pools<Real> P, int par)
{
    pdl_wait();
    using Acc = typename AccT<Real>::T;
    __shared__ unsigned s_ev[C_NCOUNT];
    Ctl *ctl = W.ctl;
    const int n = (int)min((long long)ctl->cand_n, (long long)W.cand_cap);
    const unsigned long long step = ctl->step[par];
    const int cur = ctl->cur;
    int *cellA = P.cell[cur];
    Real *offA = P.off[cur], *vxA = P.vx[cur], *vyA = P.vy[cur], *vzA = P.vz[cur];
    BirthRec<Real> *stage = reinterpret_cast<BirthRec<Real> *>(W.births);
    Acc *accG = acc_global<Real>(W);
    for (int base = blockIdx.x * COLLIDE_THREADS; base < n; base += gridDim.x * COLLIDE_THREADS) {
        for (int q = threadIdx.x; q < C_NCOUNT; q += COLLIDE_THREADS) s_ev[q] = 0;
        __syncthreads();
        const int dblk = (W.cand[base].y >> 8) / NSP;
        const int q = base + threadIdx.x;
        if (q < n) {
            const int2 e = W.cand[q];
            const int i = e.x, ds = e.y >> 8, bin = e.y & 0xFF;
            const int d = ds / NSP, s = ds % NSP;
            const Disc &Dd = W.disc[d];
            const SpeciesC &S = Dd.sp[s];
            const int rel = i - Dd.pbase[s];
            const int sub = (W.cnt[ds].chunk0 + rel / CHUNK) * SUBTILES + (rel % CHUNK) / SUBTILE;
            const int slot = rel % SUBTILE;
            int c = 0;
            Real off = Real(0);
            Real vx = vxA[i], vy = vyA[i], vz = vzA[i];
            const Real nun = S.nbins > 0 ? pick<Real>(W.nubin[S.bin_off + bin].numax_n, W.nubin[S.bin_off + bin].numax_n_f)
                                         : pick<Real>(S.numax_n, S.numax_n_f);
            const BirthSink<Real> B{stage + (size_t)sub * W.birth_cap, W.tile_cnt + (size_t)sub * NSP, ctl, W.birth_cap};
            const Outcome o = gas_collide<Real>(W, Dd, s, (unsigned)rel, step, nun, vx, vy, vz, cellA + i,
                                                offA + i, c, off, slot << 1, B);
            // a null event leaves the particle as it was: nothing to write
            if (o.alive) {
                if (o.reaction >= 0) {
                    vxA[i] = vx;
                    vyA[i] = vy;
                    vzA[i] = vz;
                }
            } else {
                cellA[i] = -1;
                deposit_global(accG + (size_t)s * W.total_nodes + Dd.gbase, c, off, -1);
            }
            if (d == dblk) {
                if (o.viol) atomicAdd(&s_ev[C_VIOL_GAS], 1u);
                if (o.reaction >= 0) atomicAdd(&s_ev[C_EVENTS + o.reaction], 1u);
            } else {
                unsigned long long *g = W.counters + (size_t)d * C_NCOUNT;
                if (o.viol) atomicAdd(&g[C_VIOL_GAS], 1ull);
                if (o.reaction >= 0) atomicAdd(&g[C_EVENTS + o.reaction], 1ull);
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < C_NCOUNT; k += COLLIDE_THREADS)
            if (s_ev[k]) atomicAdd(&W.counters[(size_t)dblk * C_NCOUNT + k], (unsigned long long)s_ev[k]);
        __syncthreads();
    }
}

// Bound on P = n dx sigma u_n n1 of channel j of species S for a particle
// of speed |v|, over every gas molecule Box-Muller can give (|V| below 10
// thermal speeds): the prefix maximum of n dx sigma u_n over the table up
// to the centre-of-mass energy of |v| + 10 v_gas (beyond the table: the last
// value times that speed), times n1, with a 1e-3 margin for rounding.  A
// draw at or above it cannot collide, whatever the molecule.
// (The speed and its place on the species' energy grid are the same for all
// channels of the species: dsmc_locate once per particle and speed,
// dsmc_bound per channel.)
template <typename Real>
__device__ __forceinline__ void dsmc_locate(const WsPtrs &W, const SpeciesC &S, const Real v[3], Real &umax,
                                            int &k, int &region)
{
    umax = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + Real(10) * pick<Real>(S.vgas_n, S.vgas_n_f);
    const XsPoint<Real> pm = xs_locate<Real>(W.tables[S.table_lo], Lut<Real>::E(W), pick<Real>(S.Ek, S.Ek_f) * umax * umax);
    k = pm.k;
    region = pm.region;
}

template <typename Real>
__device__ __forceinline__ Real dsmc_bound(const WsPtrs &W, const SpeciesC &S, int j, Real umax, int k, int region,
                                           Real n1)
{
    const Real *tb = GasTab<Real>::ptr(W) + S.gtab_off;
    const Real *pmr = GasTab<Real>::bound(W) + S.gtab_off;
    Real bnd;
    if (region == 0) {
        bnd = tb[j] * umax;
    } else if (region == 1) {
        bnd = pmr[(size_t)k * S.gtab_ld + j];
    } else {
        const Real last = tb[(size_t)(k + 1) * S.gtab_ld + j] * umax;
        const Real pmv = pmr[(size_t)k * S.gtab_ld + j];
        bnd = last > pmv ? last : pmv;
    }
    return bnd * n1 * Real(1.001);
}

// The paper's sequential scheme for the gas channels (Sec. II, Eq. 1),
// every n1 steps after the sort: part 0 walks the gas channels of the list
// numbered below (13), part 1 those above (14).  One block per tile of the
// table rebuilt after the sort; the tile's particles are held in shared
// memory and the list is walked channel by channel.  For a channel every
// particle of its species draws its test number and compares it with a
// bound on P (dsmc_bound); those below it are queued and the block's threads
// take the queue one entry each: a gas molecule from the Maxwellian, P = n
// sigma(E) u n1 dt (clamped at 1 and counted), the test, the kinematics.  A
// particle that dies in (15), (16) or (17) is replaced by its product, which
// meets the later channels ("readmitted").  Random numbers: stream 6 of the
// chain's first particle, sub-stream = the channel's place in the list,
// draws 4g (molecule), 4g + 1 (test, direction), 4g + 2 (second direction of
// (18)) in generation g.  Products are recorded in the first particle's
// sub-tile: (18)'s with product bits 0 (electron) and 1 (O2+), the one that
// ends a chain with bit 1.  The decisions are those of walking each
// particle's chain in turn: a particle's channels stay in list order, and
// particles do not interact.
template <typename Real>
__global__ void __launch_bounds__(DSMC_THREADS, 3)
k_dsmc(WsPtrs W, Pools<Real> P, int par, int part)
{
    pdl_wait();
    __shared__ unsigned s_ev[C_NCOUNT];
    __shared__ Real sv[3][CHUNK];        // velocity of the chain's current particle
    __shared__ signed char ssp[CHUNK];   // its species, -1 for no particle
    __shared__ unsigned char sgen[CHUNK];
    __shared__ unsigned short sq[CHUNK]; // queue of one channel
    __shared__ Real sumax[CHUNK];        // speed bound and grid place of the particle (dsmc_locate)
    __shared__ unsigned short sk[CHUNK];
    __shared__ unsigned char sreg[CHUNK];
    __shared__ unsigned s_qn;
    Ctl *ctl = W.ctl;
    const int chunk = blockIdx.x;
    if (chunk >= ctl->total_chunks) return;
    int lo = 0, hi = W.D * NSP;  // (discharge, species) of the tile
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (W.cnt[mid].chunk0 <= chunk) lo = mid; else hi = mid;
    }
    const int ds = lo;
    const Counts &C = W.cnt[ds];
    if (chunk >= C.chunk0 + C.nchunk) return;  // padding between species
    const int d = ds / NSP, s = ds % NSP;
    const Disc &Dd = W.disc[d];
    const int tid = threadIdx.x;
    for (int q = tid; q < C_NCOUNT; q += DSMC_THREADS) s_ev[q] = 0;
    if (part == 1 && tid < SUBTILES) W.tile_cnt[(size_t)(chunk * SUBTILES + tid) * NSP] = 0;
    if (tid == 0) s_qn = 0u;
    const unsigned long long step = ctl->step[par];
    const int cur = ctl->cur;
    int *cellA = P.cell[cur];
    Real *offA = P.off[cur], *vxA = P.vx[cur], *vyA = P.vy[cur], *vzA = P.vz[cur];
    BirthRec<Real> *stage = reinterpret_cast<BirthRec<Real> *>(W.births);
    const Real *lutE = Lut<Real>::E(W);
    const Real n1 = Real(Dd.n1);
    const int rel0 = (chunk - C.chunk0) * CHUNK;
    const int pb = Dd.pbase[s];
    unsigned nlive = 0;
    for (int local = tid; local < CHUNK; local += DSMC_THREADS) {
        const int rel = rel0 + local;
        signed char sp = -1;
        if (rel < C.n) {
            const int i = pb + rel;
            if (cellA[i] >= 0) {
                sp = (signed char)s;
                const Real v[3] = {vxA[i], vyA[i], vzA[i]};
                sv[0][local] = v[0];
                sv[1][local] = v[1];
                sv[2][local] = v[2];
                Real um;
                int k, reg;
                dsmc_locate<Real>(W, Dd.sp[s], v, um, k, reg);
                sumax[local] = um;
                sk[local] = (unsigned short)k;
                sreg[local] = (unsigned char)reg;
                ++nlive;
            }
        }
        ssp[local] = sp;
        sgen[local] = 0;
    }
    if (nlive) atomicAdd(&s_ev[C_DSMC], nlive);
    __syncthreads();
    unsigned ntest = 0;  // Eq. 1 tests of this thread's particles
    for (int kk = 0; kk < Dd.ndsmc; ++kk) {
        const DsmcCh &e = Dd.dsmc[kk];
        if (part == 0 ? e.reaction > 12 : e.reaction < 15) continue;  // uniform
        const SpeciesC &S = Dd.sp[e.sp];
        // the test of every particle of the channel's species against the
        // bound, the thread's four particles side by side (independent chains)
        {
            constexpr int PT = CHUNK / DSMC_THREADS;
            bool in[PT];
            unsigned w[PT];
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const int local = tid + q * DSMC_THREADS;
                in[q] = ssp[local] == e.sp;
                w[q] = in[q] ? rng_block(Dd.seed, Dd.discharge, s, 6, kk, 4u * sgen[local] + 1u, step,
                                         (unsigned)(rel0 + local)).x
                             : 0u;
            }
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const int local = tid + q * DSMC_THREADS;
                if (!in[q]) continue;
                ++ntest;
                if (unif<Real>(w[q]) < dsmc_bound<Real>(W, S, e.j, sumax[local], sk[local], sreg[local], n1))
                    sq[atomicAdd(&s_qn, 1u)] = (unsigned short)local;
            }
        }
        __syncthreads();
        const int nq = (int)s_qn;
        if (nq > 0) {
            const GasChan &ch = S.ch[e.j];
            for (int qi = tid; qi < nq; qi += DSMC_THREADS) {
                const int local = sq[qi];
                const int rel = rel0 + local;
                const unsigned gen = sgen[local];
                Real v[3] = {sv[0][local], sv[1][local], sv[2][local]};
                const uint4 b = rng_block(Dd.seed, Dd.discharge, s, 6, kk, 4u * gen + 1u, step, (unsigned)rel);
                const uint4 a = rng_block(Dd.seed, Dd.discharge, s, 6, kk, 4u * gen, step, (unsigned)rel);
                Real n0, nn1, n2, n3;
                box_muller<Real>(a.x, a.y, n0, nn1);
                box_muller<Real>(a.z, a.w, n2, n3);
                const Real vg = pick<Real>(S.vgas_n, S.vgas_n_f);
                const Real V[3] = {vg * n0, vg * nn1, vg * n2};
                const Real g0 = v[0] - V[0], g1 = v[1] - V[1], g2 = v[2] - V[2];
                const Real u2 = g0 * g0 + g1 * g1 + g2 * g2;
                const Real u = sqrt(u2);
                const Real E = pick<Real>(S.Ek, S.Ek_f) * u2;
                // n_j dx sigma_j(E) from the species' node-major table
                const XsPoint<Real> pt = xs_locate<Real>(W.tables[S.table_lo], lutE, E);
                const Real *ra = GasTab<Real>::ptr(W) + S.gtab_off + (size_t)pt.k * S.gtab_ld;
                const Real xa = ra[e.j], xb = ra[S.gtab_ld + e.j];
                Real xs = pt.region == 2 ? xb : xa + pt.f * (xb - xa);
                xs = E < pick<Real>(ch.th, ch.th_f) ? Real(0) : xs;
                Real Pj = xs * u * n1;
                if (Pj > Real(1)) {
                    atomicAdd(&s_ev[C_VIOL_PAIR], 1u);
                    Pj = Real(1);
                }
                if (!(unif<Real>(b.x) < Pj)) continue;
                atomicAdd(&s_ev[C_EVENTS + ch.reaction], 1u);
                Real nd[3], nd2[3] = {Real(0), Real(0), Real(1)};
                iso_dir<Real>(unif<Real>(b.y), unif<Real>(b.z), nd);
                if (ch.reaction == 18) {
                    const uint4 e2 = rng_block(Dd.seed, Dd.discharge, s, 6, kk, 4u * gen + 2u, step, (unsigned)rel);
                    iso_dir<Real>(unif<Real>(e2.x), unif<Real>(e2.y), nd2);
                }
                GasProducts<Real> pr;
                Real vo[3];
                Real um;
                int bk, breg;
                if (gas_event<Real>(W, Dd, S, ch, v, V, E, nd, nd2, vo, pr)) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) sv[q][local] = vo[q];
                    dsmc_locate<Real>(W, S, vo, um, bk, breg);
                    if (pr.n > 0) {
                        const int i = pb + rel;
                        const int sub = chunk * SUBTILES + local / SUBTILE;
                        const BirthSink<Real> B{stage + (size_t)sub * W.birth_cap, W.tile_cnt + (size_t)sub * NSP,
                                                ctl, W.birth_cap};
                        for (int q = 0; q < pr.n; ++q)
                            stage_birth<Real>(B, ((local % SUBTILE) << 1) | pr.prod[q], pr.sp[q], cellA[i], offA[i],
                                              pr.v[q]);
                    }
                } else {
                    ssp[local] = (signed char)pr.sp[0];
#pragma unroll
                    for (int q = 0; q < 3; ++q) sv[q][local] = pr.v[0][q];
                    sgen[local] = (unsigned char)(gen + 1u);
                    dsmc_locate<Real>(W, Dd.sp[pr.sp[0]], pr.v[0], um, bk, breg);
                }
                sumax[local] = um;
                sk[local] = (unsigned short)bk;
                sreg[local] = (unsigned char)breg;
            }
        }
        __syncthreads();
        if (tid == 0) s_qn = 0u;
        __syncthreads();
    }
    if (ntest) atomicAdd(&s_ev[C_PEVAL], ntest);
    // write back: the first particle's new velocity, or its removal and the
    // product that ends its chain; part 0 raises the species' recorded
    // largest speed (the particle-target pass that follows bounds P with it)
    Real m2 = Real(0);
    for (int local = tid; local < CHUNK; local += DSMC_THREADS) {
        const int rel = rel0 + local;
        if (rel >= C.n) break;
        const int i = pb + rel;
        const int c = cellA[i];
        if (c < 0) continue;
        const Real v[3] = {sv[0][local], sv[1][local], sv[2][local]};
        if (sgen[local] == 0) {
            vxA[i] = v[0];
            vyA[i] = v[1];
            vzA[i] = v[2];
            m2 = fmax(m2, Real(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
        } else {
            const Real off = offA[i];
            cellA[i] = -1;
            deposit_global(acc_global<Real>(W) + (size_t)s * W.total_nodes + Dd.gbase, c, off, -1);
            const int sub = chunk * SUBTILES + local / SUBTILE;
            const BirthSink<Real> B{stage + (size_t)sub * W.birth_cap, W.tile_cnt + (size_t)sub * NSP, ctl, W.birth_cap};
            stage_birth<Real>(B, ((local % SUBTILE) << 1) | 1, ssp[local], c, off, v);
        }
    }
    if (part == 0) vmax_raise(W.vmax2, ds, (double)m2);
    __syncthreads();
    for (int k = tid; k < C_NCOUNT; k += DSMC_THREADS)
        if (s_ev[k]) atomicAdd(&W.counters[(size_t)d * C_NCOUNT + k], (unsigned long long)s_ev[k]);
}

// Births of one step appended after the survivors, per discharge and
// product species in tile order (tiles are numbered in (parent species,
// slot) order), i.e. in parent order; their charge is deposited.  Each block
// takes BIRTHS_THREADS consecutive tiles (one per thread, coalesced counts)
// in ticket order; its place among the blocks of its discharge is the sum of
// the per-species totals that every earlier block publishes before it reads
// (all read at once by the block's threads; waits are bounded).
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <typename Real>
__global__ void __launch_bounds__(BIRTHS_THREADS)
k_births(WsPtrs W, Pools<Real> P, int par, int salt)
{
    pdl_wait();
    using Acc = typename AccT<Real>::T;
    __shared__ int wsum[NSP][BIRTHS_THREADS / 32];
    __shared__ int s_blk, s_excl[NSP], s_tot[NSP];
    __shared__ unsigned s_part[NSP][BIRTHS_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Ctl *ctl = W.ctl;
    if (tid == 0) s_blk = (int)atomicAdd(&ctl->births_ticket, 1u);
    __syncthreads();
    const int blk = s_blk;  // blocks in ticket order: all earlier ones are running or done
    const int total = ctl->total_chunks * SUBTILES;  // sub-tiles
    const int t = blk * BIRTHS_THREADS + tid;       // this thread's sub-tile
    const int tfirst_blk = blk * BIRTHS_THREADS;
    if (tfirst_blk >= total) return;
    // discharge of the block: every discharge's tiles start at a multiple of
    // BIRTHS_THREADS, so a block never spans two discharges
    int d = 0;
    {
        int lo = 0, hi = W.D;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (W.cnt[mid * NSP].chunk0 * SUBTILES <= tfirst_blk) lo = mid; else hi = mid;
        }
        d = lo;
    }
    const int T1 = (W.cnt[d * NSP + 2].chunk0 + W.cnt[d * NSP + 2].nchunk) * SUBTILES;
    int mine[NSP] = {0, 0, 0};
    const bool in = t < total && t < T1;
    const BirthRec<Real> *rec = reinterpret_cast<const BirthRec<Real> *>(W.births) + (size_t)t * W.birth_cap;
    int nrec = 0;  // records of this sub-tile (any order; the tag gives species and parent order)
    if (in) {
        nrec = min(W.tile_cnt[(size_t)t * NSP], W.birth_cap);
        for (int r = 0; r < nrec; ++r) ++mine[rec[r].tag & 3];
    }
    int excl[NSP];
#pragma unroll
    for (int q = 0; q < NSP; ++q) {
        int v = mine[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += x;
        }
        if (lane == 31) wsum[q][warp] = v;
        excl[q] = v - mine[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NSP; ++q) {
            int v = lane < BIRTHS_THREADS / 32 ? wsum[q][lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += x;
            }
            if (lane < BIRTHS_THREADS / 32) wsum[q][lane] = v;
            if (lane == 31) s_tot[q] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NSP; ++q) excl[q] += warp > 0 ? wsum[q][warp - 1] : 0;
    // this block's exclusive prefix within its discharge: the sum of the
    // aggregates that the discharge's earlier blocks publish.  Every earlier
    // block took its ticket first, so it is running or done, and it publishes
    // before it reads; all threads read the predecessors' words at once.
    // The words carry the step and which append of the step wrote them (0
    // after the collisions, 1 after the sequential gas scheme).
    {
        const unsigned long long epoch = (((ctl->step[par] + 1ull) << 1) | (unsigned)salt) & 0xFFFFFFFFull;
        const int first_blk = W.cnt[d * NSP].chunk0 * SUBTILES / BIRTHS_THREADS;
        if (tid < NSP) st_release_u64(W.births_lb + (size_t)blk * NSP + tid, (epoch << 32) | (unsigned)s_tot[tid]);
        unsigned part[NSP] = {0u, 0u, 0u};
        const int npred = (blk - first_blk) * NSP;
        long long spins = 0;
        for (int k = tid; k < npred; k += BIRTHS_THREADS) {
            const int j = first_blk + k / NSP, q = k % NSP;
            unsigned long long v = ld_acquire_u64(W.births_lb + (size_t)j * NSP + q);
            while ((v >> 32) != epoch && spins <= SPIN_LIMIT) {
                ++spins;
                __nanosleep(64);
                v = ld_acquire_u64(W.births_lb + (size_t)j * NSP + q);
            }
            if ((v >> 32) != epoch) {
                set_status(ctl, ST_TIMEOUT);
                break;
            }
            const unsigned a = (unsigned)(v & 0xFFFFFFFFull);
#pragma unroll
            for (int r = 0; r < NSP; ++r) part[r] += r == q ? a : 0u;
        }
#pragma unroll
        for (int q = 0; q < NSP; ++q) {
            const unsigned v = __reduce_add_sync(0xffffffffu, part[q]);
            if (lane == 0) s_part[q][warp] = v;
        }
        __syncthreads();
        if (tid < NSP) {
            const int q = tid;
            unsigned ex = 0;
            for (int w = 0; w < BIRTHS_THREADS / 32; ++w) ex += s_part[q][w];
            const unsigned own = (unsigned)s_tot[q];
            s_excl[q] = (int)ex;
            // the block holding the last tile of the discharge sets the counts
            if (tfirst_blk <= T1 - 1 && T1 - 1 < tfirst_blk + BIRTHS_THREADS) {
                Counts &cs = W.cnt[d * NSP + q];
                const long long nn = (long long)cs.n_snap + ex + own;
                cs.n = (int)(nn < W.disc[d].cap[q] ? nn : W.disc[d].cap[q]);
            }
        }
    }
    __syncthreads();
    if (!in || nrec == 0) return;
    const Disc &Dd = W.disc[d];
    const int cur = ctl->cur;
    Acc *accG = acc_global<Real>(W);
    // a record's place among its species: the number of that species'
    // records with a smaller tag (parent slot, then product)
    for (int r = 0; r < nrec; ++r) {
        const BirthRec<Real> &b = rec[r];
        const int q = b.tag & 3;
        int rank = 0;
        for (int k = 0; k < nrec; ++k) {
            const int tk = rec[k].tag;
            rank += (tk & 3) == q && tk < b.tag;
        }
        const long long dst = (long long)W.cnt[d * NSP + q].n_snap + s_excl[q] + excl[q] + rank;
        if (dst >= Dd.cap[q]) {
            set_status(ctl, ST_CAPACITY);
            continue;
        }
        const int g = Dd.pbase[q] + (int)dst;
        P.cell[cur][g] = b.c;
        P.off[cur][g] = b.off;
        P.vx[cur][g] = b.vx;
        P.vy[cur][g] = b.vy;
        P.vz[cur][g] = b.vz;
        deposit_global(accG + (size_t)q * W.total_nodes + Dd.gbase, b.c, b.off, 1);
    }
}

template <typename Real>
static size_t push_smem_bytes(int Nmax, int eedf_max, int fm_max, int nw, int qcap, bool cells)
{
    size_t b = sizeof(unsigned long long) * (Nmax + 2) + sizeof(Real) * (Nmax + 2);
    b += sizeof(int) * nw * qcap;  // candidate slots
    b += sizeof(unsigned) * (eedf_max + fm_max);
    b += (size_t)nw * qcap;        // candidate energy bins
    b = (b + 15) & ~size_t(15);
    if (cells) b += sizeof(unsigned) * (Nmax + 2);  // particles per cell
    return (b + 15) & ~size_t(15);
}

// The push's launch shapes (threads per block, slots per thread, blocks per
// SM the registers are sized for): the FP32 path has several for the
// autotuner, the FP64 path one.  Results do not depend on the shape (exact
// integer charge sums, births in parent order).
using PushF0 = PushShape<256, 4, 3>;
using PushF1 = PushShape<128, 4, 6>;
using PushF2 = PushShape<512, 4, 1>;
using PushF3 = PushShape<128, 8, 4>;
using PushF4 = PushShape<256, 8, 2>;
using PushD0 = PushShape<256, 4, 2>;

template <typename Real, typename SH>
static cudaError_t push_shape_setup(LaunchCfg &L, int k)
{
    const size_t sm = push_smem_bytes<Real>(L.maxN, 0, 0, SH::nw, SH::qcap, sizeof(Real) == 4);
    const size_t smd = push_smem_bytes<Real>(L.maxN, L.eedf_max, L.fm_max, SH::nw, SH::qcap, false);
    cudaError_t e = cudaFuncSetAttribute(k_push<Real, false, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_push<Real, true, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<Real, false, SH>, SH::threads, sm);
    if (e != cudaSuccess) return e;
    L.shape_threads[k] = SH::threads;
    L.shape_spt[k] = SH::spt;
    L.shape_max_per_sm[k] = per_sm < 1 ? 1 : per_sm;
    L.shape_smem[k] = sm;
    L.shape_smem_diag[k] = smd;
    return cudaSuccess;
}

cudaError_t push_configure(bool fp64, LaunchCfg &L, int num_sms)
{
    cudaError_t e;
    if (fp64) {
        L.push_nshapes = 1;
        if ((e = push_shape_setup<double, PushD0>(L, 0))) return e;
    } else {
        L.push_nshapes = 5;
        if ((e = push_shape_setup<float, PushF0>(L, 0))) return e;
        if ((e = push_shape_setup<float, PushF1>(L, 1))) return e;
        if ((e = push_shape_setup<float, PushF2>(L, 2))) return e;
        if ((e = push_shape_setup<float, PushF3>(L, 3))) return e;
        if ((e = push_shape_setup<float, PushF4>(L, 4))) return e;
    }
    L.num_sms = num_sms;
    L.push_shape = 0;
    L.push_max_per_sm = L.shape_max_per_sm[0];
    L.push_per_sm = L.push_max_per_sm;
    L.push_blocks = num_sms * L.push_per_sm;
    L.push_smem = L.shape_smem[0];
    L.push_smem_diag = L.shape_smem_diag[0];
    L.collide_blocks = num_sms * 8;
    return cudaSuccess;
}

template <typename Real, typename SH>
static void launch_push_shape(bool diag, const WsPtrs &W, const Pools<Real> &P, int par, const LaunchCfg &L,
                              cudaStream_t st)
{
    const int em = diag ? L.eedf_max : 0, fm = diag ? L.fm_max : 0;
    const size_t sm = diag ? L.push_smem_diag : L.push_smem;
    if (diag)
        launch_k(k_push<Real, true, SH>, L.push_blocks, SH::threads, sm, st, W, P, par, L.maxN, em, fm);
    else
        launch_k(k_push<Real, false, SH>, L.push_blocks, SH::threads, sm, st, W, P, par, L.maxN, em, fm);
}

cudaError_t launch_push(bool fp64, bool diag, const WsPtrs &W, const void *pools, int par,
                        const LaunchCfg &L, cudaStream_t st)
{
    if (fp64) {
        launch_push_shape<double, PushD0>(diag, W, *static_cast<const Pools<double> *>(pools), par, L, st);
    } else {
        const Pools<float> &P = *static_cast<const Pools<float> *>(pools);
        switch (L.push_shape) {
        case 1: launch_push_shape<float, PushF1>(diag, W, P, par, L, st); break;
        case 2: launch_push_shape<float, PushF2>(diag, W, P, par, L, st); break;
        case 3: launch_push_shape<float, PushF3>(diag, W, P, par, L, st); break;
        case 4: launch_push_shape<float, PushF4>(diag, W, P, par, L, st); break;
        default: launch_push_shape<float, PushF0>(diag, W, P, par, L, st); break;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_collide(bool fp64, const WsPtrs &W, const void *pools, int par, int blocks, cudaStream_t st)
{
    if (fp64)
        launch_k(k_collide<double>, blocks, COLLIDE_THREADS, 0, st, W, *static_cast<const Pools<double> *>(pools), par);
    else
        launch_k(k_collide<float>, blocks, COLLIDE_THREADS, 0, st, W, *static_cast<const Pools<float> *>(pools), par);
    return cudaGetLastError();
}

cudaError_t launch_births(bool fp64, const WsPtrs &W, const void *pools, int par, int max_blocks,
                          cudaStream_t st, int salt)
{
    if (fp64)
        launch_k(k_births<double>, max_blocks, BIRTHS_THREADS, 0, st, W, *static_cast<const Pools<double> *>(pools), par,
                 salt);
    else
        launch_k(k_births<float>, max_blocks, BIRTHS_THREADS, 0, st, W, *static_cast<const Pools<float> *>(pools), par,
                 salt);
    return cudaGetLastError();
}

cudaError_t launch_dsmc(bool fp64, const WsPtrs &W, const void *pools, int par, int part, cudaStream_t st)
{
    if (fp64)
        launch_k(k_dsmc<double>, W.max_chunks, DSMC_THREADS, 0, st, W, *static_cast<const Pools<double> *>(pools), par,
                 part);
    else
        launch_k(k_dsmc<float>, W.max_chunks, DSMC_THREADS, 0, st, W, *static_cast<const Pools<float> *>(pools), par,
                 part);
    return cudaGetLastError();
}

} // namespace o2
