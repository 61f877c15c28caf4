// o2pic_dev.cuh -- device data layout, constants and small device helpers of
// libo2pic (GB300, sm_103a).  Shared by the kernels and the host driver of the
// library; the CPU oracle does not use any of it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace o2 {

constexpr int NSP = 3;                 // 0 e, 1 O-, 2 O2+
constexpr int CHUNK = 1024;            // slots per push chunk
constexpr int SUBTILE = 128;           // slots of one warp in a tile (32 lanes x 4)
constexpr int SUBTILES = 1024 / SUBTILE;
constexpr int BIRTH_CAP_W = 32;        // births staged per sub-tile (null-collision scheme)
constexpr int BIRTH_CAP_SEQ = 128;     // the same with the sequential gas scheme (n1 steps of collisions at once)
constexpr int COLLIDE_THREADS = 256;   // threads per block of the collision kernel
#ifndef O2_TILES_PER_TICKET
#define O2_TILES_PER_TICKET 8
#endif
constexpr int TILES_PER_TICKET = O2_TILES_PER_TICKET;  // tiles taken per atomic ticket by a push block
constexpr int BIRTHS_THREADS = 512;    // block of the birth-append kernel (sub-tiles)
constexpr int TILE_ALIGN = BIRTHS_THREADS / (1024 / 128);  // tiles per birth-append block
#ifndef O2_SORT_WARPS
#define O2_SORT_WARPS 4
#endif
#ifndef O2_SORT_WARP_SLOTS
#define O2_SORT_WARP_SLOTS 8192
#endif
#ifndef O2_SORT_ILP
#define O2_SORT_ILP 8
#endif
constexpr int SORT_WARPS = O2_SORT_WARPS;  // warps per sort block
constexpr int SORT_WARP_SLOTS = O2_SORT_WARP_SLOTS;  // slots per sort warp (16-bit counters)
constexpr int SORT_ILP = O2_SORT_ILP;  // 32-slot rows loaded per warp before ranking
constexpr int SORT_CHUNK = SORT_WARPS * SORT_WARP_SLOTS;
constexpr int COLSCAN_SEG = 32;  // rows of the sort's count matrix per column-scan warp
constexpr int PAIR_BIRTH_CAP = 16;     // births of (19) per cell per pass
constexpr int MAX_GAS_CH = 16;
#ifndef O2_FIELD_THREADS
#define O2_FIELD_THREADS 1024
#endif
constexpr int FIELD_THREADS = O2_FIELD_THREADS;
constexpr int FIELD_ILP = 4;  // nodes per thread whose accumulators the field kernel loads at once
constexpr int FIX_BITS = 24;           // fixed-point deposit: weight * 2^24
constexpr int MAX_DISCHARGES = 1024;
constexpr long long SPIN_LIMIT = 1LL << 22;  // polls of a bounded wait

enum : unsigned {
    ST_CAPACITY = 1u,   // particle capacity exceeded
    ST_TIMEOUT = 2u,    // look-back wait gave up
    ST_BIRTHBUF = 4u,   // a per-chunk or per-cell birth buffer overflowed
    ST_BADSTATE = 8u,   // an impossible state was found (index out of range)
    ST_NONFINITE = 16u  // a particle's position or velocity became NaN or infinite
};

// Counters accumulated on the device (per discharge).
enum {
    C_ABS = 0,          // 6: absorbed (species*2 + wall)
    C_EVENTS = 6,       // 20: events per reaction number 0..19
    C_VIOL_GAS = 26,
    C_VIOL_PAIR = 27,
    C_SLOTS = 28,       // slots processed by the push (all species)
    C_CANDS = 29,       // null-collision candidates
    C_LIVE = 30,        // live particles pushed (particle-steps)
    C_BSLOTS = 31,      // slots of species with an energy-binned bound (vy, vz read)
    C_BCANDS = 32,      // candidates of those species
    C_COUL = 33,        // particles through the Coulomb pass (cells with >= 2 of a species)
    C_DSMC = 34,        // live slots visited by the sequential gas scheme (both parts)
    C_PEVAL = 35,       // Eq. 1 probabilities evaluated (pair-pass candidates, sequential-scheme tests)
    C_NCOUNT = 36
};

struct TableDesc {
    int off;            // offset of the nodes in the LUT arrays
    int n;              // nodes
    int reaction;
    int pad;
    double th;          // threshold [eV]
    double lnE0;        // log of the first node
    double inv_dlog;    // (n-1) / log(E_last/E_0)
    float th_f, lnE0_f, inv_dlog_f, pad_f;  // FP32 copies for the FP32 path
};

struct GasChan {
    int table;          // index into the table descriptors
    int reaction;
    double th;          // threshold [eV]
    float th_f, pad_f;
    double coef;        // n_target * dx (normalised frequency per unit u_n * sigma)
    double dloss;       // 2 dE / mu * (dt/dx)^2 (inelastic reduction of u_n^2)
    float coef_f, dloss_f;
};

// one energy bin of a collision-frequency bound
constexpr int NUBIN_MAX = 64;
constexpr int NUBIN_LOG2_E0 = -6;  // bins are quarter octaves of lab energy from 2^-6 eV
struct NuBin {
    unsigned tnull;     // null-collision threshold on a 32-bit word
    float numax_n_f;    // nu_max dt
    double numax_n;
};

struct SpeciesC {
    double qm;          // (q/m) dt^2 / dx : normalised acceleration per V/m
    double numax_n;     // nu_max * dt
    double numax;       // nu_max [1/s]
    double vgas_n;      // sqrt(kT/M_O2) * dt/dx
    double Ek;          // (1/2) mu (dx/dt)^2 / e: E_cm[eV] = Ek * u_n^2
    double mfrac;       // m/(m+M_O2)
    double Mfrac;       // M_O2/(m+M_O2)
    double ke_eV;       // (1/2) m (dx/dt)^2 / e: lab kinetic energy per u_n^2
    double vscale;      // dx/dt: normalised -> m/s
    double coul_k;      // Coulomb: <tan^2(chi/2)> u_n^3 per particle of the cell (Eq. 2)
    unsigned int tnull; // null-collision threshold on a 32-bit word
    int nch;
    int table_lo;       // first table of the shared grid (for the index)
    int gtab_ld;        // row length of the node-major gas table (multiple of 4)
    int gtab_off;       // first element of this (discharge, species) gas table
    int nbins;          // energy bins of the collision-frequency bound (0: one bound)
    int bin_off;        // first entry of this species' bins in WsPtrs::nubin
    // FP32 copies (the FP32 path never converts from FP64 on the device)
    float qm_f, numax_n_f, vgas_n_f, Ek_f, mfrac_f, Mfrac_f, ke_eV_f, coul_k_f;
    GasChan ch[MAX_GAS_CH];
};

struct PairC {          // particle-target reaction of one discharge
    int table;          // -1 = absent
    int proj, targ;
    int pad;
    double coef;        // weight * n1: P = count * coef * sigma * u_n
    double Ek;          // (1/2) mu (dx/dt)^2 / e
    double mfrac, Mfrac;// m/(m+M), M/(m+M) of the pair
    double dloss;       // 2 dE/mu (dt/dx)^2
    // bound on sigma(E) u_n over the table: sigma u_n <= max(bnd_g, bnd_s * u_n)
    // (u_n relative speed in cells per step; margins included)
    double bnd_g, bnd_s;
    float Ek_f, mfrac_f, Mfrac_f, dloss_f, coef_f, pad_f;
    float bnd_g_f, bnd_s_f;
};

// one gas channel of the sequential scheme's list (Table I order)
constexpr int MAX_DSMC = 3 * MAX_GAS_CH;
struct DsmcCh {
    int sp;        // projectile species
    int j;         // index in the species' channel list (SpeciesC::ch)
    int reaction;
    int pad;
};

struct Disc {
    int N;                   // cells
    int gbase;               // first node of this discharge in grid arrays
    int pbase[NSP];          // first slot of each species in the particle pools
    int cap[NSP];            // slots per species
    int ccell_base;          // first entry in per-cell pair arrays
    int sort_cbase[NSP];     // first entry of the sort count matrix per species
    int sort_gmax[NSP];      // sort blocks available per species
    int cs_base;             // first entry of cell_start arrays (3*(N+2) per discharge)
    double dx, dt, L, weight;
    double U_rf, omega, phase;
    double vol_fix;          // density per accumulated unit (interior node)
    double dens_fix, dens_fix_wall;  // weight / (node volume * 2^FIX_BITS), inside / at walls
    double Kfix;             // e weight 2^-FIX_BITS / eps0
    double kE;               // dt^2/dx
    double f15, mu2_15;      // reaction (15) product speed factor
    double f16;              // (16): v_e = |v_Om| * f16
    double f17;              // (17): w = sqrt(E_cm * f17)
    double eedf_scale, iedf_scale, fm_scale, fm_emax;
    float f15_f, f16_f, f17_f, eedf_scale_f, iedf_scale_f, fm_scale_f, fm_emax_f, pad_f;
    int eedf_bins, iedf_bins, fm_bins, fm_xbins;
    int diag_every, n1, sort_interval, n2;
    int eedf_base, iedf_base, fm_base, pad2;
    unsigned long long seed;
    int discharge;
    int cx_iso;
    int gas_scheme;          // 0 null collision, 1 the sequential channel list every n1 steps
    int ion_sub;             // ions pushed on steps n = 0 mod ion_sub (1: every step)
    int coul_inter;          // inter-species Coulomb collisions after the intra-species ones
    // inter-species Coulomb, pairs e-O-, e-O2+, O- - O2+: <tan^2(chi/2)> u_n^3 per
    // particle of the less numerous species in the cell, and each member's
    // share of the change of g (m_other / (m_a + m_b))
    double ci_k[3], ci_frac[3][2];
    float ci_k_f[3], ci_frac_f[3][2], pad_ci;
    int ndsmc;               // gas channels of the sequential list
    DsmcCh dsmc[MAX_DSMC];   // in the order of Table I
    SpeciesC sp[NSP];
    PairC pair[3];           // 13, 14, 19
};

struct Ctl {
    unsigned long long step[2];   // step number, read by parity
    unsigned int status;
    int cur;                      // particle buffer holding the state (0/1)
    unsigned int ticket;          // dynamic chunk counter of the push
    int total_chunks;             // chunks in the current push
    int D;                        // discharges
    unsigned int births_ticket;   // block order of the birth-append kernel
    unsigned int cand_n;          // collision candidates listed by the push this step
    unsigned int colscan_ticket;  // warp order of the sort's column scan
    unsigned int sort_epoch;      // sorts so far (tags the column scan's words)
};

// Per (discharge, species) dynamic counts.
struct Counts {
    int n;          // slots in use (live + dead not yet compacted)
    int n_snap;     // slots at the start of the current push
    int chunk0;     // first chunk of this (d, s) in the current push
    int nchunk;
};

// Pointers to every array of the workspace (device addresses).
template <typename Real>
struct Pools {
    int *cell[2];
    Real *off[2], *vx[2], *vy[2], *vz[2];
};

struct WsPtrs {
    Ctl *ctl;
    Disc *disc;
    Counts *cnt;              // [D*3]
    int *chunk_ds;            // [D*3 + 1] first chunk per (d,s) (prefix), device copy
    int *tile_cnt;            // [max_chunks * SUBTILES * 3] births per sub-tile and product species
    void *births;             // [max_chunks * SUBTILES * birth_cap] staged birth records
    int birth_cap;            // records per sub-tile
    unsigned long long *colscan_agg;  // column totals of the sort's row segments, tagged with the sort
    unsigned long long *births_lb;  // [max_chunks * SUBTILES / BIRTHS_THREADS * 3] look-back words
    unsigned long long *acc_fix;  // [3 * total_nodes] fixed-point density accumulators
    double *acc_dbl;          // [3 * total_nodes] FP64 accumulators
    double *Efield;           // [total_nodes] E [V/m]
    void *Ereal;              // [total_nodes] E as Real for the push
    double *phi;              // [total_nodes]
    double *rho;              // [total_nodes]
    double *dens;             // [3 * total_nodes]
    double *dens_sum;         // [3 * total_nodes] (FP64 path)
    double *phi_sum;          // [total_nodes] (FP64 path)
    long long *dens_sum_fix;  // same memory as dens_sum: exact fixed-point sums (FP32 path)
    __int128 *phi_s2_sum;     // [total_nodes] sums of S2_{i-1} (FP32 path)
    double *phi0_sum, *D0_sum;// [D] sums of phi_0 and D0 (FP32 path)
    unsigned long long *nsamp;// [D]
    unsigned long long *counters; // [D * C_NCOUNT]
    unsigned int *eedf, *iedf, *fm;
    TableDesc *tables;
    double *lutE, *lutS;      // FP64 nodes and values
    float *lutEf, *lutSf;     // FP32 copies
    double *gtab;             // node-major gas tables: n_j dx sigma_j(E_k), [k][j] per (d, s)
    float *gtabf;
    double *gpm;              // same layout: bound on n_j dx sigma_j(E) u_n for E up to E_{k+1}
    float *gpmf;
    int *sort_counts;         // count matrix
    unsigned short *sort_whist;  // per-warp bucket counts of each sort block: [(block, warp), bucket]
    int *cell_start;          // [sum over d of 3*(N+2)]
    int *sort_live;           // [D*3]
    int *sort_tot;            // [sum over d of 3*(N+2)] slots per bucket
    int *pair_bcount;         // [total cells] births of (19) per cell
    int *cell_disc;           // [total cells] discharge of each global cell
    int *pair_first;          // [total cells] first flagged projectile of the current reaction
    unsigned long long *vmax2;// [D * 3] largest speed^2 (cells/step, double bits): at the last
                              // sort, raised by the velocity changes since (Coulomb pass, first
                              // part of the sequential gas scheme); the particle-target pass's cap
    struct NuBin *nubin;      // [D * NUBIN_MAX] electron collision-frequency bounds per energy bin
    int2 *cand;               // [cand_cap] collision candidates: (slot, ds << 8 | energy bin)
    int cand_cap;
    int *pair_kills;          // [total cells * 3] particles killed per species in this pass
    void *pair_births;        // [total cells * PAIR_BIRTH_CAP] records
    int total_nodes;
    int total_cells;
    int max_chunks;
    int D;
};

// FP64 constant for the FP64 path, its FP32 copy for the FP32 path
template <typename Real> __device__ __forceinline__ Real pick(double d, float f);
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }

// ---------------------------------------------------------------- Philox

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies words 0 and 2 by the round multipliers, swaps the halves and
// xors in the round key; the key advances by the Weyl increments between
// rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        unsigned lo0 = 0xD2511F53u * c.x;
        unsigned hi0 = __umulhi(0xD2511F53u, c.x);
        unsigned lo1 = 0xCD9E8D57u * c.z;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z);
        uint4 n;
        n.x = hi1 ^ c.y ^ k.x;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k.y;
        n.w = lo0;
        c = n;
    }
    return c;
}

// Counter layout (identical to the oracle's contract): word 0 = step low 32
// bits, word 1 = index, word 2 = stream<<28 | sub<<20 | draw, word 3 =
// discharge<<16 | species<<8 | step bits 32..39; key = seed (low, high).
__device__ __forceinline__ uint4 rng_block(unsigned long long seed, int disc, int sp,
                                           int stream, int sub, unsigned draw,
                                           unsigned long long step, unsigned index)
{
    uint4 c;
    c.x = (unsigned)(step & 0xFFFFFFFFull);
    c.y = index;
    c.z = ((unsigned)stream << 28) | ((unsigned)sub << 20) | (draw & 0xFFFFFu);
    c.w = ((unsigned)disc << 16) | ((unsigned)sp << 8) | (unsigned)((step >> 32) & 0xFF);
    uint2 k = make_uint2((unsigned)(seed & 0xFFFFFFFFull), (unsigned)(seed >> 32));
    return philox10(c, k);
}

template <typename Real> __device__ __forceinline__ Real unif(unsigned w);
template <> __device__ __forceinline__ double unif<double>(unsigned w)
{
    return ((double)w + 0.5) * (1.0 / 4294967296.0);
}
// FP32: (2k+1) 2^-24 with k = w >> 9, exactly representable, inside (0, 1);
// within 2^-24 of the FP64 value.
template <> __device__ __forceinline__ float unif<float>(unsigned w)
{
    return (float)(w >> 9) * (1.0f / 8388608.0f) + (1.0f / 16777216.0f);
}

__device__ __forceinline__ void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincospi_(float x, float *s, float *c) { sincospif(x, s, c); }

template <typename Real>
__device__ __forceinline__ void box_muller(unsigned a, unsigned b, Real &n0, Real &n1)
{
    Real r = sqrt(Real(-2) * log(unif<Real>(a)));
    Real s, c;
    sincospi_(Real(2) * unif<Real>(b), &s, &c);
    n0 = r * c;
    n1 = r * s;
}

template <typename Real>
__device__ __forceinline__ void iso_dir(Real r1, Real r2, Real n[3])
{
    Real cx = Real(1) - Real(2) * r1;
    Real sx = Real(1) - cx * cx;
    sx = sx > Real(0) ? sqrt(sx) : Real(0);
    Real s, c;
    sincospi_(Real(2) * r2, &s, &c);
    n[0] = sx * c;
    n[1] = sx * s;
    n[2] = cx;
}

// Kernels of a time step are launched with programmatic dependent launch:
// the next kernel may be scheduled while the previous one drains, and waits
// here, before it reads anything, until that one has completed (a no-op
// when launched without the attribute).
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// a sub-cycled ion species rests (is not pushed) at this step
__device__ __forceinline__ bool species_rests(const Disc &Dd, int s, unsigned long long step)
{
    return s > 0 && Dd.ion_sub > 1 && step % (unsigned long long)Dd.ion_sub != 0ull;
}

__device__ __forceinline__ void set_status(Ctl *ctl, unsigned bits)
{
    atomicOr(&ctl->status, bits);
}

// Raise the recorded largest speed^2 of (discharge, species) ds to the
// warp's largest m2 (every lane of the warp calls it; non-negative doubles
// order like their bit patterns).
__device__ __forceinline__ void vmax_raise(unsigned long long *vmax2, int ds, double m2)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    if ((threadIdx.x & 31) == 0 && m2 > 0.0)
        atomicMax(&vmax2[ds], (unsigned long long)__double_as_longlong(m2));
}

} // namespace o2
