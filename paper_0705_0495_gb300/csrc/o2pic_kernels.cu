// o2pic_kernels.cu -- field solve, cell sort, particle-target pass, load and
// deposit kernels of libo2pic (GB300, sm_103a).
#include "o2pic_launch.h"

namespace o2 {

constexpr double QE_ = 1.602176634e-19;
constexpr double EPS0_ = 8.8541878128e-12;

// ------------------------------------------------------------ helpers

template <typename Real> struct AccK;
template <> struct AccK<float> {
    using T = unsigned long long;
    static __device__ __forceinline__ T *ptr(const WsPtrs &W) { return W.acc_fix; }
};
template <> struct AccK<double> {
    using T = double;
    static __device__ __forceinline__ T *ptr(const WsPtrs &W) { return W.acc_dbl; }
};

__device__ __forceinline__ void dep_global(unsigned long long *acc, int c, float off, int sign)
{
    unsigned w1 = __float2uint_rn(off * (float)(1 << FIX_BITS));
    unsigned w0 = (1u << FIX_BITS) - w1;
    unsigned long long a = w0, b = w1;
    if (sign < 0) { a = 0ull - a; b = 0ull - b; }
    atomicAdd(&acc[c], a);
    atomicAdd(&acc[c + 1], b);
}
__device__ __forceinline__ void dep_global(double *acc, int c, double off, int sign)
{
    atomicAdd(&acc[c], sign * (1.0 - off));
    atomicAdd(&acc[c + 1], sign * off);
}

__device__ __forceinline__ double acc_to_weight(unsigned long long a)
{
    return (double)(long long)a * (1.0 / (double)(1 << FIX_BITS));
}
__device__ __forceinline__ double acc_to_weight(double a) { return a; }

// inclusive scan of x[0..M) in shared memory by one block (deterministic order)
template <int NT>
__device__ void block_scan_inclusive(double *x, int M, double *warp_tot)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (M + NT - 1) / NT;
    const int lo = tid * per, hi = min(M, lo + per);
    double run = 0.0;
    for (int i = lo; i < hi; ++i) {
        run += x[i];
        x[i] = run;
    }
    // exclusive scan of the thread totals
    double v = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = lane < NT / 32 ? warp_tot[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < NT / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    double excl = v - run + (warp > 0 ? warp_tot[warp - 1] : 0.0);
    for (int i = lo; i < hi; ++i) x[i] += excl;
    __syncthreads();
}

// exclusive scan of a[0..M) in shared memory by one block; returns the total
__device__ int block_scan_exclusive_int(int *a, int M, int *wsum)
{
    const int NT = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (M + NT - 1) / NT;
    const int lo = tid * per, hi = min(M, lo + per);
    int run = 0;
    for (int i = lo; i < hi; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    int v = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < NT / 32) wsum[lane] = w;
    }
    __syncthreads();
    const int excl = v - run + (warp > 0 ? wsum[warp - 1] : 0);
    for (int i = lo; i < hi; ++i) a[i] += excl;
    const int total = wsum[NT / 32 - 1];
    __syncthreads();
    return total;
}

// ------------------------------------------------------------ field

// Per discharge (one block): densities from the accumulators, Poisson with
// phi_0 = U_rf sin(2 pi f t + phase), phi_N = 0, and the node field.
// The tridiagonal system (phi_{i-1} - 2 phi_i + phi_{i+1}) = -rho_i dx^2/eps0
// is solved exactly by two prefix sums: with s_i = rho_i dx^2/eps0,
// S1_i = sum_{k<=i} s_k and S2_i = sum_{m<=i} S1_m (i >= 1),
// phi_i = phi_0 + i D0 - S2_{i-1}, D0 fixed by phi_N = 0.
__device__ void tile_table(const WsPtrs &W, int par, unsigned long long step, bool advance);

template <typename Real>
__global__ void __launch_bounds__(FIELD_THREADS)
k_field(WsPtrs W, int par, int diag, int mode)
{
    pdl_wait();
    extern __shared__ __align__(16) double fsm[];
    __shared__ double warp_tot[FIELD_THREADS / 32];
    __shared__ double s_rho0, s_rhoN, s_D0;
    using Acc = typename AccK<Real>::T;
    const int d = blockIdx.x;
    const Disc &Dd = W.disc[d];
    const int N = Dd.N, g = Dd.gbase, tid = threadIdx.x;
    Ctl *ctl = W.ctl;
    const unsigned long long step = ctl->step[par];
    const int tn = W.total_nodes;
    const double dx = Dd.dx;
    // the drive's potential, once per block by one thread: GB300 runs FP64 on
    // few units, and 1024 threads each evaluating sin() would cost more than
    // the whole solve
    __shared__ double s_phi0;
    auto drive = [&]() { return Dd.U_rf * sin(Dd.omega * ((double)step * Dd.dt) + Dd.phase); };
    double phi0;
    Real *Er = reinterpret_cast<Real *>(W.Ereal) + g;
    Acc *acc = AccK<Real>::ptr(W);
    if constexpr (sizeof(Real) == 4) {
        // FP32 path: the accumulators are exact fixed-point sums (weight *
        // 2^FIX_BITS).  With q_i the net charge in these units and
        // K = e w 2^-FIX_BITS / eps0: interior s_i = K dx q_i, S1 = prefix
        // sums of q (exact int64), S2 = prefix sums of S1 (exact int128), and
        //   phi_i = phi_0 + i D0 - K dx S2_{i-1},  D0 = (K dx S2_{N-1} - phi_0)/N
        //   E_i = (K/2) (T_i - T0),  T0 = 2 D0 / (K dx), with the integers
        //   T_i = S1_i + S1_{i-1} inside, T_0 = -2 q_0, T_N = 2 (S1_{N-1} + q_N)
        // (the wall values are Gauss's law on the half cells).  T_i - round(T0)
        // is exact, so E leaves FP64 only through O(1) constants.
        long long *S1 = reinterpret_cast<long long *>(fsm);  // N+1 entries
        __shared__ long long wl[FIELD_THREADS / 32];
        __shared__ __int128 w128[FIELD_THREADS / 32];
        __shared__ long long s_q0, s_qN, s_T0i;
        __shared__ float s_hKf, s_frf;
        __shared__ int s_intE;
        const double K = Dd.Kfix;  // e w 2^-FIX_BITS / eps0
        const bool full = diag || mode != 0;
        // the accumulators of FIELD_ILP nodes per thread are all loaded before
        // any is cleared, so that their loads are in flight together (a store
        // to one could otherwise alias the next load, one latency each)
        bool clear[NSP];
#pragma unroll
        for (int s = 0; s < NSP; ++s) clear[s] = mode == 0 && !species_rests(Dd, s, step);
        for (int i0 = tid; i0 <= N; i0 += FIELD_THREADS * FIELD_ILP) {
            long long aa[FIELD_ILP][NSP];
#pragma unroll
            for (int j = 0; j < FIELD_ILP; ++j) {
                const int i = i0 + j * FIELD_THREADS;
#pragma unroll
                for (int s = 0; s < NSP; ++s) aa[j][s] = i <= N ? (long long)acc[(size_t)s * tn + g + i] : 0;
            }
            // thread 0 evaluates the drive while its loads are in flight
            if (tid == 0 && i0 == 0) s_phi0 = drive();
#pragma unroll
            for (int j = 0; j < FIELD_ILP; ++j) {
                const int i = i0 + j * FIELD_THREADS;
                if (i > N) break;
                const long long *a = aa[j];
#pragma unroll
                for (int s = 0; s < NSP; ++s) {
                    const size_t k = (size_t)s * tn + g + i;
                    if (clear[s]) acc[k] = Acc(0);
                    if (diag) W.dens_sum_fix[k] += a[s];  // exact sums; scaled at read-out
                }
                const long long q = a[2] - a[0] - a[1];
                S1[i] = (i == 0 || i == N) ? 0 : q;
                if (i == 0) s_q0 = q;
                if (i == N) s_qN = q;
                if (full) {
                    const double sc = (i == 0 || i == N) ? Dd.dens_fix_wall : Dd.dens_fix;
#pragma unroll
                    for (int s = 0; s < NSP; ++s) W.dens[(size_t)s * tn + g + i] = (double)a[s] * sc;
                    W.rho[g + i] = QE_ * (double)q * sc;
                }
            }
        }
        __syncthreads();
        phi0 = s_phi0;
        // inclusive int64 scan of S1[1..N-1] and the int128 sum of the result
        const int M = N - 1, lane = tid & 31, warp = tid >> 5;
        const int per = (M + FIELD_THREADS - 1) / FIELD_THREADS;
        const int lo = 1 + tid * per, hi = min(N, lo + per);
        long long run = 0;
        for (int i = lo; i < hi; ++i) {
            run += S1[i];
            S1[i] = run;
        }
        long long v = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long x = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += x;
        }
        if (lane == 31) wl[warp] = v;
        __syncthreads();
        if (warp == 0) {
            long long w = lane < FIELD_THREADS / 32 ? wl[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long x = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += x;
            }
            if (lane < FIELD_THREADS / 32) wl[lane] = w;
        }
        __syncthreads();
        const long long excl = v - run + (warp > 0 ? wl[warp - 1] : 0);
        __int128 part = 0;
        for (int i = lo; i < hi; ++i) {
            S1[i] += excl;
            part += (__int128)S1[i];
        }
        // inclusive int128 scan of the thread parts (the total is S2_{N-1})
        __int128 pv = part;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long lo_ = __shfl_up_sync(0xffffffffu, (unsigned long long)pv, o);
            const long long hi_ = __shfl_up_sync(0xffffffffu, (long long)(pv >> 64), o);
            if (lane >= o) pv += ((__int128)hi_ << 64) | (__int128)lo_;
        }
        if (lane == 31) w128[warp] = pv;
        __syncthreads();
        if (tid == 0) {
            __int128 r = 0;
            for (int w = 0; w < FIELD_THREADS / 32; ++w) {
                r += w128[w];
                w128[w] = r;
            }
            const double D0 = (K * dx * (double)r - phi0) / (double)N;
            s_D0 = D0;
            const double T0 = 2.0 * D0 / (K * dx);
            s_intE = (K > 0.0 && fabs(T0) < 4.0e18) ? 1 : 0;
            const long long T0i = s_intE ? llround(T0) : 0;
            s_T0i = T0i;
            s_hKf = (float)(0.5 * K);
            s_frf = (float)(T0 - (double)T0i);
            if (diag) {
                W.phi0_sum[d] += phi0;
                W.D0_sum[d] += D0;
            }
        }
        __syncthreads();
        const long long T0i = s_T0i;
        const float hKf = s_hKf, frf = s_frf;
        const bool intE = s_intE != 0;
        for (int i = tid; i <= N; i += FIELD_THREADS) {
            const long long Ti = (i == 0) ? -2 * s_q0 : (i == N ? 2 * (S1[N - 1] + s_qN) : S1[i] + S1[i - 1]);
            if (intE) {
                Er[i] = hKf * (__ll2float_rn(Ti - T0i) - frf);
                if (full) W.Efield[g + i] = 0.5 * K * ((double)(Ti - T0i) - (double)frf);
            } else {  // no charge or an extreme field: evaluate in FP64
                const double E = -s_D0 / dx + 0.5 * K * (double)Ti;
                Er[i] = (Real)E;
                if (full) W.Efield[g + i] = E;
            }
        }
        const double D0 = s_D0;
        if (full) {
            // potential and the exact running sums of S2 for its average
            const __int128 before = (warp > 0 ? w128[warp - 1] : (__int128)0) + pv - part;
            __int128 r = before;
            for (int i = lo; i < hi; ++i) {
                // r = S2_{i-1} when node i is reached
                double p = phi0 + (double)i * D0 - K * dx * (double)r;
                if (diag) W.phi_s2_sum[g + i] += r;
                W.phi[g + i] = p;
                r += (__int128)S1[i];
            }
            if (tid == 0) W.phi[g] = phi0;
            if (tid == 0) W.phi[g + N] = 0.0;
        }
    } else {
        if (tid == 0) s_phi0 = drive();
        __syncthreads();
        phi0 = s_phi0;
        double *x = fsm;  // N+1 entries
        for (int i = tid; i <= N; i += FIELD_THREADS) {
            const double vol = (i == 0 || i == N) ? 0.5 * dx : dx;
            const double scale = Dd.weight / vol;
            double dn[NSP];
#pragma unroll
            for (int s = 0; s < NSP; ++s) {
                const size_t k = (size_t)s * tn + g + i;
                dn[s] = acc_to_weight(acc[k]) * scale;
                if (mode == 0 && !species_rests(Dd, s, step)) acc[k] = Acc(0);
                W.dens[k] = dn[s];
                if (diag) W.dens_sum[k] += dn[s];
            }
            const double rho = QE_ * (dn[2] - dn[0] - dn[1]);
            W.rho[g + i] = rho;
            if (i == 0) s_rho0 = rho;
            if (i == N) s_rhoN = rho;
            x[i] = rho * dx * dx / EPS0_;
        }
        __syncthreads();
        // scans over interior nodes 1..N-1, stored at x[1..N-1]
        const int M = N - 1;
        if (M > 0) {
            block_scan_inclusive<FIELD_THREADS>(x + 1, M, warp_tot);  // S1
            block_scan_inclusive<FIELD_THREADS>(x + 1, M, warp_tot);  // S2
        }
        if (tid == 0) s_D0 = M > 0 ? (-phi0 + x[M]) / (double)N : -phi0 / (double)N;
        __syncthreads();
        const double D0 = s_D0;
        double *phi = W.phi + g;
        for (int i = tid; i <= N; i += FIELD_THREADS) {
            double p;
            if (i == 0) p = phi0;
            else if (i == N) p = 0.0;
            else p = phi0 + (double)i * D0 - (i >= 2 ? x[i - 1] : 0.0);
            phi[i] = p;
        }
        __syncthreads();
        for (int i = tid; i <= N; i += FIELD_THREADS) {
            double E;
            if (i == 0) E = -(phi[1] - phi[0]) / dx - s_rho0 * dx / (2.0 * EPS0_);
            else if (i == N) E = -(phi[N] - phi[N - 1]) / dx + s_rhoN * dx / (2.0 * EPS0_);
            else E = -(phi[i + 1] - phi[i - 1]) / (2.0 * dx);
            W.Efield[g + i] = E;
            Er[i] = (Real)E;
            if (diag) W.phi_sum[g + i] += phi[i];
        }
    }
    if (diag && tid == 0) W.nsamp[d] += 1ull;
    if (mode != 0 || blockIdx.x != 0) return;
    // block 0: tile table of this step's push and the step counter
    __syncthreads();
    tile_table(W, par, step, true);
}

// Tile table of the current counts: tiles of each discharge start at a
// multiple of TILE_ALIGN, so that the birth-append blocks (BIRTHS_THREADS
// sub-tiles) never span two, and those of each species at a multiple of
// TILES_PER_TICKET, so that a push ticket never spans two; the birth counts
// of the padding tiles after each species (never pushed) are cleared.  With
// `advance` the next step's counter is set and the candidate list emptied.
__device__ void tile_table(const WsPtrs &W, int par, unsigned long long step, bool advance)
{
    Ctl *ctl = W.ctl;
    const int tid = threadIdx.x;
    if (tid == 0) {
        // tiles of each discharge start at a multiple of TILE_ALIGN, so that the
        // birth-append blocks (BIRTHS_THREADS sub-tiles) never span two, and
        // those of each species at a multiple of TILES_PER_TICKET, so that a
        // push ticket never spans two
        int chunk = 0;
        for (int ds = 0; ds < W.D * NSP; ++ds) {
            Counts &C = W.cnt[ds];
            if (ds % NSP == 0) chunk = (chunk + TILE_ALIGN - 1) / TILE_ALIGN * TILE_ALIGN;
            else chunk = (chunk + TILES_PER_TICKET - 1) / TILES_PER_TICKET * TILES_PER_TICKET;
            C.n_snap = C.n;
            C.chunk0 = chunk;
            C.nchunk = (C.n + CHUNK - 1) / CHUNK;
            chunk += C.nchunk;
        }
        if (chunk > W.max_chunks) {
            set_status(ctl, ST_CAPACITY);
            chunk = 0;
        }
        ctl->total_chunks = chunk;
        ctl->ticket = 0u;
        ctl->births_ticket = 0u;
        if (advance) {
            ctl->cand_n = 0u;
            ctl->step[par ^ 1] = step + 1ull;
        }
    }
    __syncthreads();
    for (int ds = 0; ds < W.D * NSP; ++ds) {
        const Counts &C = W.cnt[ds];
        const int t0 = C.chunk0 + C.nchunk;
        const int t1 = (t0 + TILES_PER_TICKET - 1) / TILES_PER_TICKET * TILES_PER_TICKET;
        const int n = (t1 - t0) * SUBTILES * NSP;
        for (int k = tid; k < n; k += blockDim.x) W.tile_cnt[(size_t)t0 * SUBTILES * NSP + k] = 0;
    }
}

__global__ void __launch_bounds__(256) k_retile(WsPtrs W, int par)
{
    pdl_wait();
    tile_table(W, par, 0ull, false);
}

// ------------------------------------------------------------- sort

// block -> (ds, index of the block within ds) from a host-built table
__device__ __forceinline__ void sort_block(const int *tab, int &ds, int &bi)
{
    ds = tab[2 * blockIdx.x];
    bi = tab[2 * blockIdx.x + 1];
}

// Histogram of cells (dead slots in bucket N) of one block of SORT_CHUNK
// slots, one per warp (SORT_WARP_SLOTS slots, 16-bit counts): the warps'
// rows go to sort_whist for the scatter, their sum to row bi of the
// (block x bucket) count matrix of ds.  Each warp reads SORT_ILP slots per
// lane before counting, to keep loads in flight.
template <typename Real>
__global__ void __launch_bounds__(SORT_WARPS * 32)
k_sort_count(WsPtrs W, Pools<Real> P, const int *tab)
{
    pdl_wait();
    extern __shared__ __align__(16) unsigned short wsm[];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // the column scan that follows: its warp order and the tag of its words
        W.ctl->colscan_ticket = 0u;
        W.ctl->sort_epoch += 1u;
    }
    int ds, bi;
    sort_block(tab, ds, bi);
    const int d = ds / NSP, s = ds % NSP;
    const Disc &Dd = W.disc[d];
    const int N = Dd.N, n = W.cnt[ds].n;
    const int G = (n + SORT_CHUNK - 1) / SORT_CHUNK;
    if (bi == 0 && threadIdx.x == 0) W.vmax2[ds] = 0ull;  // raised by the scatter
    if (bi >= G) return;
    const int stride = (N + 2) & ~1;
    for (int i = threadIdx.x; i < SORT_WARPS * stride; i += blockDim.x) wsm[i] = 0;
    __syncthreads();
    const int *cell = P.cell[W.ctl->cur] + Dd.pbase[s];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned short *hw = wsm + (size_t)w * stride;
    const int lo = bi * SORT_CHUNK + w * SORT_WARP_SLOTS;
    const int hi = min(n, lo + SORT_WARP_SLOTS);
    for (int i0 = lo; i0 < hi; i0 += 32 * SORT_ILP) {
        int b[SORT_ILP];
#pragma unroll
        for (int r = 0; r < SORT_ILP; ++r) {
            const int i = i0 + r * 32 + lane;
            b[r] = -1;
            if (i < hi) {
                const int c = cell[i];
                b[r] = c < 0 ? N : c;
            }
        }
#pragma unroll
        for (int r = 0; r < SORT_ILP; ++r) {
            // sorted runs: a whole row in one bucket needs no match
            const int b0 = __shfl_sync(0xffffffffu, b[r], 0);
            if (__all_sync(0xffffffffu, b[r] == b0)) {
                if (lane == 0 && b0 >= 0) hw[b0] += (unsigned short)32;
                __syncwarp();
                continue;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, b[r]);
            if (b[r] >= 0 && lane == __ffs(peers) - 1) hw[b[r]] += (unsigned short)__popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    int *row = W.sort_counts + Dd.sort_cbase[s] + (size_t)bi * (N + 1);
    unsigned short *wrow = W.sort_whist + ((size_t)Dd.sort_cbase[s] + (size_t)bi * (N + 1)) * SORT_WARPS;
    for (int i = threadIdx.x; i <= N; i += blockDim.x) {
        int t = 0;
#pragma unroll
        for (int q = 0; q < SORT_WARPS; ++q) {
            const unsigned short h = wsm[(size_t)q * stride + i];
            wrow[(size_t)q * (N + 1) + i] = h;
            t += h;
        }
        row[i] = t;
    }
}

// Column scan of the (block x bucket) count matrix: running sums down the
// sort blocks, so that each (block, bucket) entry becomes that block's first
// slot inside the bucket, and the bucket totals in sort_tot.  One warp per
// (d, s, 32 consecutive buckets, COLSCAN_SEG consecutive rows), in the order
// of a ticket: the warp loads its rows (each row's 32 buckets in one 128-byte
// load), publishes their column totals tagged with the sort, adds those of
// the earlier row segments of its buckets (warps with smaller tickets, so
// running or done, which publish before they wait) and writes each entry's
// exclusive prefix; the segment holding the last row writes the totals.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(256)
k_sort_colscan(WsPtrs W, const int *unit_base)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    Ctl *ctl = W.ctl;
    int u = 0;
    if (lane == 0) u = (int)atomicAdd(&ctl->colscan_ticket, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    const int nds = W.D * NSP;
    if (u >= unit_base[nds]) return;
    int lo = 0, hi = nds;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (unit_base[mid] <= u) lo = mid; else hi = mid;
    }
    const int ds = lo;
    const int d = ds / NSP, s = ds % NSP;
    const Disc &Dd = W.disc[d];
    const int N = Dd.N;
    const int n = W.cnt[ds].n;
    const int G = (n + SORT_CHUNK - 1) / SORT_CHUNK;
    const int nseg = (Dd.sort_gmax[s] + COLSCAN_SEG - 1) / COLSCAN_SEG;
    const int local = u - unit_base[ds];
    const int grp = local / nseg, sg = local % nseg;
    const int c = grp * 32 + lane;
    const bool valid = c <= N;
    int *cnt = W.sort_counts + Dd.sort_cbase[s];
    const int r0 = sg * COLSCAN_SEG;
    int v[COLSCAN_SEG];
    unsigned tot = 0;
#pragma unroll
    for (int k = 0; k < COLSCAN_SEG; ++k) {
        const int r = r0 + k;
        v[k] = (valid && r < G) ? cnt[(size_t)r * (N + 1) + c] : 0;
        tot += (unsigned)v[k];
    }
    const unsigned long long epoch = ctl->sort_epoch;
    // the words of segments 0 .. nseg-1 of this bucket group, 32 per segment
    unsigned long long *agg = W.colscan_agg + (size_t)(u - sg) * 32;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(agg + (size_t)sg * 32 + lane),
                 "l"((epoch << 32) | tot) : "memory");
    unsigned pre = 0;
    long long spins = 0;
    bool late = false;
    for (int k0 = 0; k0 < sg && !late; k0 += 8) {
        unsigned long long w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = k0 + k < sg ? ld_relaxed_u64(agg + (size_t)(k0 + k) * 32 + lane) : 0ull;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k0 + k >= sg) break;
            while ((w[k] >> 32) != (epoch & 0xFFFFFFFFull) && spins <= SPIN_LIMIT) {
                ++spins;
                __nanosleep(64);
                w[k] = ld_relaxed_u64(agg + (size_t)(k0 + k) * 32 + lane);
            }
            if ((w[k] >> 32) != (epoch & 0xFFFFFFFFull)) {
                set_status(ctl, ST_TIMEOUT);
                late = true;
                break;
            }
            pre += (unsigned)(w[k] & 0xFFFFFFFFull);
        }
    }
    unsigned run = pre;
#pragma unroll
    for (int k = 0; k < COLSCAN_SEG; ++k) {
        const int r = r0 + k;
        if (valid && r < G) cnt[(size_t)r * (N + 1) + c] = (int)run;
        run += (unsigned)v[k];
    }
    const int last = G > 0 ? (G - 1) / COLSCAN_SEG : 0;
    if (valid && sg == last) W.sort_tot[Dd.cs_base + s * (N + 2) + c] = (int)run;
}

// Per (d, s): bucket starts (cell_start) by a scan over the bucket totals.
__global__ void __launch_bounds__(512)
k_sort_cellscan(WsPtrs W)
{
    pdl_wait();
    extern __shared__ __align__(16) int isx[];
    __shared__ int wsum[32];
    const int ds = blockIdx.x;
    const int d = ds / NSP, s = ds % NSP;
    const Disc &Dd = W.disc[d];
    const int N = Dd.N, n = W.cnt[ds].n;
    const int *tot_g = W.sort_tot + Dd.cs_base + s * (N + 2);
    int *tot = isx;  // N+1
    for (int c = threadIdx.x; c <= N; c += blockDim.x) tot[c] = n > 0 ? tot_g[c] : 0;
    __syncthreads();
    block_scan_exclusive_int(tot, N + 1, wsum);
    int *cs = W.cell_start + Dd.cs_base + s * (N + 2);
    for (int c = threadIdx.x; c <= N; c += blockDim.x) cs[c] = tot[c];
    if (threadIdx.x == 0) {
        cs[N + 1] = n;
        W.sort_live[ds] = tot[N];  // live slots = start of the dead bucket
    }
}

// Stable scatter: warp w of block bi owns slots [lo + w*SORT_WARP_SLOTS, ...);
// the per-warp bucket counts (16-bit) that the count kernel kept give each
// warp its first slot per bucket relative to the block's, then each warp
// walks its slots in order, ranking equal buckets inside a 32-slot row by
// lane.  Dead slots (bucket N) are
// dropped.  SORT_ILP rows are loaded before they are ranked.
template <typename Real>
__global__ void __launch_bounds__(SORT_WARPS * 32)
k_sort_scatter(WsPtrs W, Pools<Real> P, const int *tab)
{
    pdl_wait();
    extern __shared__ __align__(16) unsigned short hsm[];
    int ds, bi;
    sort_block(tab, ds, bi);
    const int d = ds / NSP, s = ds % NSP;
    const Disc &Dd = W.disc[d];
    const int N = Dd.N, n = W.cnt[ds].n;
    const int G = (n + SORT_CHUNK - 1) / SORT_CHUNK;
    if (bi >= G) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int stride = (N + 2) & ~1;
    unsigned short *hw = hsm + (size_t)w * stride;
    const int cur = W.ctl->cur, nxt = cur ^ 1;
    const int pb = Dd.pbase[s];
    const int *cell = P.cell[cur] + pb;
    const int lo = bi * SORT_CHUNK + w * SORT_WARP_SLOTS;
    const int hi = min(n, lo + SORT_WARP_SLOTS);
    // per bucket: warp offsets relative to the block's first slot in it, from
    // the warps' counts that the count kernel kept
    const unsigned short *wrow = W.sort_whist + ((size_t)Dd.sort_cbase[s] + (size_t)bi * (N + 1)) * SORT_WARPS;
    for (int c = threadIdx.x; c <= N; c += blockDim.x) {
        unsigned run = 0;
#pragma unroll
        for (int q = 0; q < SORT_WARPS; ++q) {
            const unsigned t = wrow[(size_t)q * (N + 1) + c];
            hsm[(size_t)q * stride + c] = (unsigned short)run;
            run += t;
        }
    }
    __syncthreads();
    const int *base = W.sort_counts + Dd.sort_cbase[s] + (size_t)bi * (N + 1);
    const int *cstart = W.cell_start + Dd.cs_base + s * (N + 2);
    const Real *offS = P.off[cur] + pb, *vxS = P.vx[cur] + pb, *vyS = P.vy[cur] + pb,
               *vzS = P.vz[cur] + pb;
    int *cellD = P.cell[nxt] + pb;
    Real *offD = P.off[nxt] + pb, *vxD = P.vx[nxt] + pb, *vyD = P.vy[nxt] + pb,
         *vzD = P.vz[nxt] + pb;
    const unsigned lt = (1u << lane) - 1u;
    // largest speed^2 of the live particles this lane moves, in the
    // particles' own precision (one conversion at the end: FP64 arithmetic
    // per particle is slow on this part)
    Real vm2 = Real(0);
    for (int i0 = lo; i0 < hi; i0 += 32 * SORT_ILP) {
        int b[SORT_ILP];
        int dst[SORT_ILP];
#pragma unroll
        for (int r = 0; r < SORT_ILP; ++r) {
            const int i = i0 + r * 32 + lane;
            b[r] = -1;
            if (i < hi) {
                const int c = cell[i];
                b[r] = c < 0 ? N : c;
            }
        }
        // every load of the rows' data (read-only path) before the ranks are
        // worked out, so that their latency overlaps that work; the source
        // and destination arrays never overlap
        Real ro[SORT_ILP], rx[SORT_ILP], ry[SORT_ILP], rz[SORT_ILP];
        int gb[SORT_ILP];
#pragma unroll
        for (int r = 0; r < SORT_ILP; ++r) {
            gb[r] = 0;
            if (b[r] >= 0 && b[r] < N) {
                const int i = i0 + r * 32 + lane;
                gb[r] = __ldg(&cstart[b[r]]) + __ldg(&base[b[r]]);
                ro[r] = __ldg(&offS[i]);
                rx[r] = __ldg(&vxS[i]);
                ry[r] = __ldg(&vyS[i]);
                rz[r] = __ldg(&vzS[i]);
            }
        }
#pragma unroll
        for (int r = 0; r < SORT_ILP; ++r) {
            dst[r] = -1;
            const int b0 = __shfl_sync(0xffffffffu, b[r], 0);
            if (__all_sync(0xffffffffu, b[r] == b0)) {
                // a whole row in one bucket: ranks are the lanes
                if (b0 >= 0 && b0 < N) dst[r] = (int)hw[b0] + lane;
                __syncwarp();
                if (lane == 0 && b0 >= 0) hw[b0] += (unsigned short)32;
                __syncwarp();
                continue;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, b[r]);
            if (b[r] >= 0 && b[r] < N) dst[r] = (int)hw[b[r]] + __popc(peers & lt);
            __syncwarp();
            if (b[r] >= 0 && lane == __ffs(peers) - 1) hw[b[r]] += (unsigned short)__popc(peers);
            __syncwarp();
        }
#pragma unroll
        for (int r = 0; r < SORT_ILP; ++r) {
            if (dst[r] >= 0) {
                const int g = gb[r] + dst[r];
                vm2 = fmax(vm2, Real(rx[r] * rx[r] + ry[r] * ry[r] + rz[r] * rz[r]));
                cellD[g] = b[r];
                offD[g] = ro[r];
                vxD[g] = rx[r];
                vyD[g] = ry[r];
                vzD[g] = rz[r];
            }
        }
    }
    // speed bound of the species for the particle-target pass
    vmax_raise(W.vmax2, ds, (double)vm2);
}

__global__ void k_sort_finish(WsPtrs W)
{
    pdl_wait();
    for (int ds = threadIdx.x; ds < W.D * NSP; ds += blockDim.x) W.cnt[ds].n = W.sort_live[ds];
    __syncthreads();
    if (threadIdx.x == 0) W.ctl->cur ^= 1;
}

// ------------------------------------------------------------ pair pass

template <typename Real>
struct PairBirth {
    int c;
    int pad;
    Real off, vx, vy, vz;
};

template <typename Real>
__device__ __forceinline__ Real pair_sigma(const WsPtrs &W, const TableDesc &T, Real E);

template <>
__device__ __forceinline__ float pair_sigma<float>(const WsPtrs &W, const TableDesc &T, float E)
{
    if (E < T.th_f) return 0.f;
    const float *nd = W.lutEf + T.off, *sv = W.lutSf + T.off;
    const int n = T.n;
    if (!(E > nd[0])) return sv[0];
    if (E >= nd[n - 1]) return sv[n - 1];
    int k = (int)((logf(E) - T.lnE0_f) * T.inv_dlog_f);
    k = k < 0 ? 0 : (k > n - 2 ? n - 2 : k);
    while (k > 0 && E < nd[k]) --k;
    while (k < n - 2 && E >= nd[k + 1]) ++k;
    const float f = (E - nd[k]) / (nd[k + 1] - nd[k]);
    return sv[k] + f * (sv[k + 1] - sv[k]);
}
template <>
__device__ __forceinline__ double pair_sigma<double>(const WsPtrs &W, const TableDesc &T, double E)
{
    if (E < T.th) return 0.0;
    const double *nd = W.lutE + T.off, *sv = W.lutS + T.off;
    const int n = T.n;
    if (!(E > nd[0])) return sv[0];
    if (E >= nd[n - 1]) return sv[n - 1];
    int k = (int)((log(E) - T.lnE0) * T.inv_dlog);
    k = k < 0 ? 0 : (k > n - 2 ? n - 2 : k);
    while (k > 0 && E < nd[k]) --k;
    while (k < n - 2 && E >= nd[k + 1]) ++k;
    const double f = (E - nd[k]) / (nd[k + 1] - nd[k]);
    return sv[k] + f * (sv[k + 1] - sv[k]);
}

template <typename Real>
__device__ __forceinline__ void iso_n(Real r1, Real r2, Real n[3])
{
    iso_dir<Real>(r1, r2, n);
}

constexpr int NO_FLAG = 0x7F7F7F7F;  // larger than any slot index

// Particle-target reaction k (0: (13), 1: (14), 2: (19)) evaluated for every
// projectile at once, as if it were the first of its cell: a random target
// of the cell (walking past dead ones), P = n_target sigma(E) u n1 dt (Eq. 1)
// with n_target from the live target count at the start of the reaction's
// pass, and the acceptance draw.  Nothing is changed here; the smallest
// projectile index of a cell that collides, finds no live target, or has
// P > 1 is recorded, and the sequential pass of that cell restarts there.
// Before it, every projectile's outcome is exactly that of the sequential
// pass, because no earlier projectile of the cell changed anything.
// Particle-target reaction k by thinning (Eq. 1): no pair of the pass is
// faster than the sum of the two species' largest speeds (recorded at the
// sort and raised by the velocity changes since), so with u_cap that sum,
// rounded up to 5 significant bits in m/s (the same grid point whatever the
// rounding of the sum), B = n_target max sigma u tau over u <= u_cap bounds P
// for every pair; the cell's candidates are its projectiles at geometric
// gaps of rate B (a random stream per cell), and a candidate reacts with
// probability min(P, 1) / min(B, 1); with B >= 1 every projectile is a
// candidate.  Every projectile then reacts with probability min(P, 1).
__device__ __forceinline__ double round_up_5bits(double u)
{
    if (!(u > 0.0)) return 0.0;
    int e;
    const double m = frexp(u, &e);
    return ldexp(ceil(m * 32.0) / 32.0, e);
}
__device__ __forceinline__ double pair_bound_B(const WsPtrs &W, const Disc &Dd, int d, const PairC &pc, int liveT)
{
    const double vs = Dd.sp[0].vscale;  // cells per step -> m/s
    const double vp = sqrt(__longlong_as_double((long long)W.vmax2[d * NSP + pc.proj]));
    const double vt = sqrt(__longlong_as_double((long long)W.vmax2[d * NSP + pc.targ]));
    const double ucap_n = round_up_5bits((vp + vt) * vs) / vs;
    return (double)liveT * pc.coef * fmax(pc.bnd_g, pc.bnd_s * ucap_n);
}
// gap before the next candidate: floor(ln U / ln(1 - B)) for the draw-th word
// of the cell's stream (B < 1, lq = ln(1 - B)), at most 2^30
__device__ __forceinline__ long long pair_gap(const Disc &Dd, int ps, int rx, unsigned draw,
                                              unsigned long long step, int c, double lq)
{
    const uint4 g = rng_block(Dd.seed, Dd.discharge, ps, 4, rx, draw, step, (unsigned)c);
    const double G = floor(log(unif<double>(g.x)) / lq);
    return G < 1073741824.0 ? (long long)G : 1073741824LL;
}

// One thread per cell: does reaction k have a candidate in it?
template <typename Real>
__global__ void __launch_bounds__(256)
k_pair_eval(WsPtrs W, Pools<Real> P, int par, int k)
{
    pdl_wait();
    const int gw = blockIdx.x * blockDim.x + threadIdx.x;
    if (gw >= W.total_cells) return;
    const int d = W.cell_disc[gw];
    const Disc &Dd = W.disc[d];
    const PairC &pc = Dd.pair[k];
    if (pc.table < 0) return;
    const int ps = pc.proj, pt = pc.targ, N = Dd.N, c = gw - Dd.ccell_base;
    const int *cs = W.cell_start + Dd.cs_base;
    const int p0 = cs[ps * (N + 2) + c], p1 = cs[ps * (N + 2) + c + 1];
    if (p1 <= p0) return;
    const int range = cs[pt * (N + 2) + c + 1] - cs[pt * (N + 2) + c];
    if (range <= 0) return;
    const int liveT = range - W.pair_kills[(size_t)gw * NSP + pt];
    if (liveT <= 0) return;
    const double B = pair_bound_B(W, Dd, d, pc, liveT);
    long long first = 0;
    if (B < 1.0) {
        const int rx = k == 0 ? 13 : (k == 1 ? 14 : 19);
        first = pair_gap(Dd, ps, rx, 0u, W.ctl->step[par], c, log1p(-B));
    }
    if (first < (long long)(p1 - p0)) W.pair_first[gw] = p0 + (int)first;
}

// Sequential pass of reaction k over one flagged cell (one warp), from its
// first flagged projectile on: projectiles in slot order, a batch of 32
// evaluated in parallel, the first accepting lane executed, the later lanes
// evaluated again.  Kills, (19)'s scattering and its births happen here.
template <typename Real>
__global__ void __launch_bounds__(256)
k_pair_fix(WsPtrs W, Pools<Real> P, int par, int k)
{
    pdl_wait();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= W.total_cells) return;
    const int first = W.pair_first[gw];
    if (first == NO_FLAG) return;
    const int d = W.cell_disc[gw];
    const Disc &Dd = W.disc[d];
    const int N = Dd.N, c = gw - Dd.ccell_base;
    const int cur = W.ctl->cur;
    const unsigned long long step = W.ctl->step[par];
    const int *cs = W.cell_start + Dd.cs_base;
    int *cellA = P.cell[cur];
    Real *offA = P.off[cur], *vxA = P.vx[cur], *vyA = P.vy[cur], *vzA = P.vz[cur];
    typename AccK<Real>::T *acc = AccK<Real>::ptr(W);
    PairBirth<Real> *births = reinterpret_cast<PairBirth<Real> *>(W.pair_births) + (size_t)gw * PAIR_BIRTH_CAP;
    unsigned long long *cnt = W.counters + (size_t)d * C_NCOUNT;
    int *kills = W.pair_kills + (size_t)gw * NSP;
    int nb = W.pair_bcount[gw];
    const int rx = k == 0 ? 13 : (k == 1 ? 14 : 19);
    const PairC &pc = Dd.pair[k];
    const int ps = pc.proj, pt = pc.targ;
    const int p0 = cs[ps * (N + 2) + c], p1 = cs[ps * (N + 2) + c + 1];
    const int t0 = cs[pt * (N + 2) + c], t1 = cs[pt * (N + 2) + c + 1];
    const int range = t1 - t0;
    const int liveT = range - kills[pt];
    const TableDesc &T = W.tables[pc.table];
    const Real coefP = Real(liveT) * pick<Real>(pc.coef, pc.coef_f);
    const int pbp = Dd.pbase[ps], pbt = Dd.pbase[pt];
    // candidates of the thinning, 32 at a time: each lane draws its gap, a
    // warp scan of (1 + gap) places them (the gaps do not depend on events)
    const double B = pair_bound_B(W, Dd, d, pc, liveT);
    const bool thin = B < 1.0;
    const double lq = thin ? log1p(-B) : 0.0;
    const Real Bc = thin ? Real(B) : Real(1);
    long long pos = p0 - 1;  // last candidate placed (warp-uniform)
    unsigned draw = 0;
    bool stop = false;
    unsigned nviol = 0, neval = 0;
    int nkp = 0, nkt = 0;
    (void)first;
    while (!stop && pos + 1 < p1) {
        long long inc = 1 + (thin ? pair_gap(Dd, ps, rx, draw + (unsigned)lane, step, c, lq) : 0LL);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += x;
        }
        const long long ipos = pos + inc;
        const int i = ipos < p1 ? (int)ipos : p1;  // p1: no candidate for this lane
        pos = __shfl_sync(0xffffffffu, ipos, 31);
        draw += 32;
        int from = 0;
        for (;;) {
            bool ev = false, ex = false, viol = false, evald = false;
            int j = -1;
            uint4 d0 = make_uint4(0, 0, 0, 0);
            if (i < p1 && lane >= from && cellA[pbp + i] >= 0) {
                d0 = rng_block(Dd.seed, Dd.discharge, ps, 2, rx, 0, step, (unsigned)i);
                j = t0 + (int)__umulhi(d0.x, (unsigned)range);
                int walked = 0;
                while (cellA[pbt + j] < 0 && walked < range) {
                    j = (j + 1 < t1) ? j + 1 : t0;
                    ++walked;
                }
                if (cellA[pbt + j] < 0) {
                    ex = true;
                } else {
                    const Real g0 = vxA[pbp + i] - vxA[pbt + j];
                    const Real g1 = vyA[pbp + i] - vyA[pbt + j];
                    const Real g2 = vzA[pbp + i] - vzA[pbt + j];
                    const Real u2 = g0 * g0 + g1 * g1 + g2 * g2;
                    const Real u = sqrt(u2);
                    const Real E = pick<Real>(pc.Ek, pc.Ek_f) * u2;
                    Real Pc = coefP * pair_sigma<Real>(W, T, E) * u;
                    if (Pc > Real(1)) {  // Eq. 1 beyond 1: clamped and counted (R10)
                        viol = true;
                        Pc = Real(1);
                    }
                    ev = unif<Real>(d0.y) * Bc < Pc;
                    evald = true;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, ev || ex);
            const int l = m ? __ffs(m) - 1 : 32;
            nviol += __popc(__ballot_sync(0xffffffffu, viol && lane <= l));
            neval += __popc(__ballot_sync(0xffffffffu, evald && lane <= l));
            if (!m) break;
            const bool exl = __shfl_sync(0xffffffffu, ex, l);
            if (exl) {
                stop = true;  // no live target left for this projectile
                break;
            }
            if (lane == l) {
                const int gi = pbp + i, gj = pbt + j;
                atomicAdd(&cnt[C_EVENTS + rx], 1ull);
                typename AccK<Real>::T *acc_p = acc + (size_t)ps * W.total_nodes + Dd.gbase;
                typename AccK<Real>::T *acc_t = acc + (size_t)pt * W.total_nodes + Dd.gbase;
                if (rx != 19) {
                    cellA[gi] = -1;
                    dep_global(acc_p, c, offA[gi], -1);
                } else {
                    uint4 d1 = rng_block(Dd.seed, Dd.discharge, ps, 2, 19, 1, step, (unsigned)i);
                    Real v[3] = {vxA[gi], vyA[gi], vzA[gi]};
                    Real V[3] = {vxA[gj], vyA[gj], vzA[gj]};
                    Real nd[3], n2[3], v1[3], Vo[3];
                    iso_n<Real>(unif<Real>(d0.z), unif<Real>(d0.w), nd);
                    const Real mf = pick<Real>(pc.mfrac, pc.mfrac_f), Mf = pick<Real>(pc.Mfrac, pc.Mfrac_f);
                    Real g0 = v[0] - V[0], g1 = v[1] - V[1], g2 = v[2] - V[2];
                    Real uu = g0 * g0 + g1 * g1 + g2 * g2 - pick<Real>(pc.dloss, pc.dloss_f);
                    Real up = uu > Real(0) ? sqrt(uu) : Real(0);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        Real vcm = mf * v[q] + Mf * V[q];
                        v1[q] = vcm + Mf * up * nd[q];
                        Vo[q] = vcm - mf * up * nd[q];
                    }
                    iso_n<Real>(unif<Real>(d1.x), unif<Real>(d1.y), n2);
                    Real e2[3] = {Vo[0], Vo[1], Vo[2]};
                    Real a0 = v1[0] - e2[0], a1 = v1[1] - e2[1], a2 = v1[2] - e2[2];
                    Real ue = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        Real cc = Real(0.5) * (v1[q] + e2[q]);
                        v1[q] = cc + Real(0.5) * ue * n2[q];
                        e2[q] = cc - Real(0.5) * ue * n2[q];
                    }
                    vxA[gi] = v1[0];
                    vyA[gi] = v1[1];
                    vzA[gi] = v1[2];
                    if (nb < PAIR_BIRTH_CAP) {
                        PairBirth<Real> &pbr = births[nb];
                        pbr.c = c;
                        pbr.off = offA[gi];
                        pbr.vx = e2[0];
                        pbr.vy = e2[1];
                        pbr.vz = e2[2];
                    } else {
                        set_status(W.ctl, ST_BIRTHBUF);
                    }
                }
                cellA[gj] = -1;
                dep_global(acc_t, c, offA[gj], -1);
            }
            __syncwarp();
            __threadfence_block();
            if (rx == 19) {
                ++nb;
                ++nkt;
            } else {
                ++nkp;
                ++nkt;
            }
            from = l + 1;
            if (from >= 32) break;
        }
    }
    if (lane == 0) {
        if (nviol) atomicAdd(&cnt[C_VIOL_PAIR], (unsigned long long)nviol);
        if (neval) atomicAdd(&cnt[C_PEVAL], (unsigned long long)neval);
        kills[ps] += nkp;
        kills[pt] += nkt;
        W.pair_bcount[gw] = nb < PAIR_BIRTH_CAP ? nb : PAIR_BIRTH_CAP;
        W.pair_first[gw] = NO_FLAG;
    }
}

// ------------------------------------------------------------ Coulomb (1)-(3)

// Arithmetic of the Coulomb collision.  FP64: correctly rounded functions.
// FP32: the hardware approximations (rsqrtf, __fdividef, __logf, __sincosf,
// each documented within a few units of 2^-22), whose errors change a
// velocity by far less than the FP32 path's tolerance of 1e-5 of the thermal
// speed; sin and cos of 2 pi r come from pi (2 r - 1) in [-pi, pi) with the
// signs of both flipped.
template <typename Real> struct CoulMath;
template <> struct CoulMath<double> {
    static __device__ __forceinline__ double inv_u32(double kn_sqrt, double u2, double u)
    {
        (void)kn_sqrt;
        return 1.0 / (u2 * u);
    }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ void normal2(unsigned a, unsigned b, double &n0, double &n1)
    {
        box_muller<double>(a, b, n0, n1);
    }
    static __device__ __forceinline__ void sincos2pi(double r, double *s, double *c) { sincospi(2.0 * r, s, c); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
};
template <> struct CoulMath<float> {
    static __device__ __forceinline__ float inv_u32(float, float u2, float u)
    {
        (void)u2;
        const float r = rsqrtf(u);
        return r * r * r * r * r * r;  // u^-3
    }
    static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
    static __device__ __forceinline__ void normal2(unsigned a, unsigned b, float &n0, float &n1)
    {
        const float x = -2.0f * __logf(unif<float>(a));
        const float r = x * rsqrtf(x);
        float s, c;
        __sincosf(3.14159265358979f * (2.0f * unif<float>(b) - 1.0f), &s, &c);
        n0 = -r * c;
        n1 = -r * s;
    }
    static __device__ __forceinline__ void sincos2pi(float r, float *s, float *c)
    {
        __sincosf(3.14159265358979f * (2.0f * r - 1.0f), s, c);
        *s = -*s;
        *c = -*c;
    }
    static __device__ __forceinline__ float sqrt_(float x) { return x * rsqrtf(x); }
};

// One binary Coulomb collision of two like particles i, j (Sec. III A, the
// model of Takizuka and Abe): tan(chi/2) = sqrt(kn / u^3) * xi with kn the
// Eq. 2 variance times u^3 for this cell, xi a standard normal; the azimuth
// phi = 2 pi r is measured from the plane of g and the z axis (the x-y plane
// when g is along z).  Each particle takes half of the change of g.
template <typename Real>
__device__ __forceinline__ void coulomb_pair(Real *vx, Real *vy, Real *vz, int i, int j, Real kn,
                                             Real xi, unsigned wphi)
{
    using M = CoulMath<Real>;
    const Real g0 = vx[i] - vx[j], g1 = vy[i] - vy[j], g2 = vz[i] - vz[j];
    const Real u2 = g0 * g0 + g1 * g1 + g2 * g2;
    if (!(u2 > Real(0))) return;
    const Real u = M::sqrt_(u2);
    const Real d = M::sqrt_(kn * M::inv_u32(Real(0), u2, u)) * xi;  // tan(chi/2)
    Real sn, om;                                                     // sin(chi), 1 - cos(chi)
    if (fabs(d) <= Real(1)) {
        const Real r = M::rcp(Real(1) + d * d);
        sn = Real(2) * d * r;
        om = Real(2) * d * d * r;
    } else {                                  // the same in 1/d (finite for any d)
        const Real e = M::rcp(d);
        const Real r = M::rcp(Real(1) + e * e);
        sn = Real(2) * e * r;
        om = Real(2) * r;
    }
    Real sp, cp;
    M::sincos2pi(unif<Real>(wphi), &sp, &cp);
    const Real up2 = g0 * g0 + g1 * g1;
    Real d0, d1, d2;
    if (up2 > Real(0)) {
        const Real up = M::sqrt_(up2), rp = M::rcp(up);
        const Real ex = g0 * rp, ey = g1 * rp;
        const Real a = g2 * sn * cp, b = u * sn * sp;
        d0 = ex * a - ey * b - g0 * om;
        d1 = ey * a + ex * b - g1 * om;
        d2 = -up * sn * cp - g2 * om;
    } else {
        d0 = u * sn * cp;
        d1 = u * sn * sp;
        d2 = -g2 * om;
    }
    vx[i] += Real(0.5) * d0;
    vy[i] += Real(0.5) * d1;
    vz[i] += Real(0.5) * d2;
    vx[j] -= Real(0.5) * d0;
    vy[j] -= Real(0.5) * d1;
    vz[j] -= Real(0.5) * d2;
}

// random numbers of collision k of a cell's pass: stream 5, the draw
// counter split over the sub-stream (high bits) and draw fields
__device__ __forceinline__ uint4 coulomb_rng(unsigned long long seed, int disc, int s,
                                             unsigned long long step, int c, unsigned k)
{
    return rng_block(seed, disc, s, 5, (int)(k >> 20), k & 0xFFFFFu, step, (unsigned)c);
}

// Copy n values of each component, COUL_COPY elements per thread in flight.
constexpr int COUL_COPY = 4;
template <typename Real>
__device__ __forceinline__ void coulomb_copy(Real *__restrict__ dx, Real *__restrict__ dy, Real *__restrict__ dz,
                                             const Real *__restrict__ sx, const Real *__restrict__ sy,
                                             const Real *__restrict__ sz, int n)
{
    for (int k0 = threadIdx.x; k0 < n; k0 += COUL_COPY * COUL_THREADS) {
        Real ax[COUL_COPY], ay[COUL_COPY], az[COUL_COPY];
#pragma unroll
        for (int q = 0; q < COUL_COPY; ++q) {
            const int k = k0 + q * COUL_THREADS;
            if (k < n) {
                ax[q] = sx[k];
                ay[q] = sy[k];
                az[q] = sz[k];
            }
        }
#pragma unroll
        for (int q = 0; q < COUL_COPY; ++q) {
            const int k = k0 + q * COUL_THREADS;
            if (k < n) {
                dx[k] = ax[q];
                dy[k] = ay[q];
                dz[k] = az[q];
            }
        }
    }
}

// largest speed^2 among n velocities (a block-strided share per thread)
template <typename Real>
__device__ __forceinline__ double speed2_max(const Real *x, const Real *y, const Real *z, int n)
{
    Real m = Real(0);
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        m = fmax(m, Real(x[k] * x[k] + y[k] * y[k] + z[k] * z[k]));
    return (double)m;
}

// Collision k of a cell with the random numbers of draw 1 + k/2: the normal
// is the first (k even) or second (k odd) of the Box-Muller pair, the
// azimuth word 2 or 3.
template <typename Real>
__device__ __forceinline__ void coulomb_one(Real *vx, Real *vy, Real *vz, int i, int j, Real kn,
                                            unsigned long long seed, int disc, int s,
                                            unsigned long long step, int c, unsigned k)
{
    const uint4 w = coulomb_rng(seed, disc, s, step, c, 1u + (k >> 1));
    Real n0, n1;
    CoulMath<Real>::normal2(w.x, w.y, n0, n1);
    coulomb_pair<Real>(vx, vy, vz, i, j, kn, (k & 1u) ? n1 : n0, (k & 1u) ? w.w : w.z);
}

// The collisions of one cell.  Thread t takes collisions 2q and 2q + 1 for
// q = t, t + T, ..., which share one draw: pi(4q) = (b + q (4a mod n)) mod n,
// advanced by T (4a mod n) mod n per iteration; pi(4q+2) = pi(4q) + 2a mod
// n and pi(k+1) = pi(k) + a mod n.  prm holds a, b, 2a mod n and 4a mod n.
template <typename Real>
__device__ __forceinline__ void coulomb_cell_pairs(Real *vx, Real *vy, Real *vz, unsigned un,
                                                   const unsigned *prm, Real kn, unsigned long long seed,
                                                   int disc, int s, unsigned long long step, int c)
{
    using M = CoulMath<Real>;
    const unsigned a = prm[0], b = prm[1], a2 = prm[2], a4 = prm[3];
    const unsigned pairs = (un & 1u) ? (un - 3u) / 2u : un / 2u;
    const unsigned t = threadIdx.x;
    unsigned x = un <= (1u << 22) ? (b + (t * a4) % un) % un
                                  : (unsigned)(((unsigned long long)t * a4 + b) % un);
    const unsigned stepA = (unsigned)(((unsigned long long)COUL_THREADS * a4) % un);
    for (unsigned q = t; 2u * q < pairs; q += COUL_THREADS) {
        const uint4 w = coulomb_rng(seed, disc, s, step, c, 1u + q);
        Real n0, n1;
        M::normal2(w.x, w.y, n0, n1);
        unsigned y = x + a;
        if (y >= un) y -= un;
        coulomb_pair<Real>(vx, vy, vz, (int)x, (int)y, kn, n0, w.z);
        if (2u * q + 1u < pairs) {
            unsigned x1 = x + a2;
            if (x1 >= un) x1 -= un;
            unsigned y1 = x1 + a;
            if (y1 >= un) y1 -= un;
            coulomb_pair<Real>(vx, vy, vz, (int)x1, (int)y1, kn, n1, w.w);
        }
        x += stepA;
        if (x >= un) x -= un;
    }
    if ((un & 1u) && t == 0) {
        const int A = (int)(((unsigned long long)a * (un - 3u) + b) % un);
        const int B = (int)(((unsigned long long)a * (un - 2u) + b) % un);
        const int C = (int)(((unsigned long long)a * (un - 1u) + b) % un);
        const Real kh = Real(0.5) * kn;
        coulomb_one<Real>(vx, vy, vz, A, B, kh, seed, disc, s, step, c, pairs);
        coulomb_one<Real>(vx, vy, vz, B, C, kh, seed, disc, s, step, c, pairs + 1u);
        coulomb_one<Real>(vx, vy, vz, C, A, kh, seed, disc, s, step, c, pairs + 2u);
    }
}

// Coulomb pass of one species in one cell per block, right after the sort
// (every slot of the cell is live).  Blocks run the O2+ cells first, then
// O-, then electrons (the largest cells first).  The n particles are paired
// by the affine permutation pi(k) = (a k + b) mod n, a coprime to n, from
// draw 0 of the cell's stream 5; collision m is (pi(2m), pi(2m+1)) with the
// random numbers of draw 1 + m/2 (two collisions per draw); for odd n thread
// 0 then runs the triangle of the last three, (A, B), (B, C), (C, A), with
// half the time each.  The pairs are disjoint, so no ordering is needed
// between threads.  A cell of at most `cap` particles is staged in shared
// memory (coalesced copies in and out); a larger one is worked on in place.
template <typename Real>
__global__ void __launch_bounds__(COUL_THREADS, 2)
k_coulomb(WsPtrs W, Pools<Real> P, int par, int cap)
{
    pdl_wait();
    extern __shared__ __align__(16) unsigned char coul_smem[];
    const int gw = blockIdx.x % W.total_cells, s = NSP - 1 - (int)(blockIdx.x / W.total_cells);
    const int d = W.cell_disc[gw];
    const Disc &Dd = W.disc[d];
    const int N = Dd.N, c = gw - Dd.ccell_base;
    const int *cs = W.cell_start + Dd.cs_base;
    const int p0 = cs[s * (N + 2) + c], p1 = cs[s * (N + 2) + c + 1];
    const int n = p1 - p0;
    if (n < 2) return;
    if (n >= (1 << 29)) {
        if (threadIdx.x == 0) set_status(W.ctl, ST_BADSTATE);
        return;
    }
    if (threadIdx.x == 0) atomicAdd(&W.counters[(size_t)d * C_NCOUNT + C_COUL], (unsigned long long)n);
    const unsigned long long step = W.ctl->step[par];
    const unsigned long long seed = Dd.seed;
    const int disc = Dd.discharge;
    const int cur = W.ctl->cur;
    const int base = Dd.pbase[s] + p0;
    Real *gx = P.vx[cur] + base, *gy = P.vy[cur] + base, *gz = P.vz[cur] + base;
    const unsigned un = (unsigned)n;
    __shared__ unsigned prm[4];  // a, b, 2a mod n, 4a mod n of the cell's permutation
    if (threadIdx.x == 0) {
        const uint4 w0 = coulomb_rng(seed, disc, s, step, c, 0u);
        unsigned a = 1u + w0.x % (un - 1u);
        for (;;) {  // a -> a mod (n-1) + 1 until coprime; a = 1 always is
            unsigned x = a, y = un;
            while (y) {
                const unsigned t = x % y;
                x = y;
                y = t;
            }
            if (x == 1u) break;
            a = a % (un - 1u) + 1u;
        }
        prm[0] = a;
        prm[1] = w0.y % un;
        prm[2] = (unsigned)((2ull * a) % un);
        prm[3] = (unsigned)((4ull * a) % un);
    }
    const SpeciesC &S = Dd.sp[s];
    const Real kn = pick<Real>(S.coul_k, S.coul_k_f) * Real(n);
    // the new speeds raise the species' recorded largest speed, which bounds
    // P in a particle-target pass of the same step
    double m2;
    if (n <= cap) {
        Real *sx = reinterpret_cast<Real *>(coul_smem), *sy = sx + cap, *sz = sy + cap;
        coulomb_copy<Real>(sx, sy, sz, gx, gy, gz, n);
        __syncthreads();
        coulomb_cell_pairs<Real>(sx, sy, sz, un, prm, kn, seed, disc, s, step, c);
        __syncthreads();
        coulomb_copy<Real>(gx, gy, gz, sx, sy, sz, n);
        m2 = speed2_max<Real>(sx, sy, sz, n);
    } else {
        __syncthreads();
        coulomb_cell_pairs<Real>(gx, gy, gz, un, prm, kn, seed, disc, s, step, c);
        __syncthreads();
        m2 = speed2_max<Real>(gx, gy, gz, n);
    }
    vmax_raise(W.vmax2, d * NSP + s, m2);
}

// One Coulomb collision between particles a (velocity va) and b (vb) of
// unlike species: as coulomb_pair, with the pair's kn, a taking fa of the
// change of g = va - vb and b minus fb of it.
template <typename Real>
__device__ __forceinline__ void coulomb_pair_ab(Real va[3], Real vb[3], Real kn, Real fa, Real fb, Real xi,
                                                unsigned wphi)
{
    using M = CoulMath<Real>;
    const Real g0 = va[0] - vb[0], g1 = va[1] - vb[1], g2 = va[2] - vb[2];
    const Real u2 = g0 * g0 + g1 * g1 + g2 * g2;
    if (!(u2 > Real(0))) return;
    const Real u = M::sqrt_(u2);
    const Real d = M::sqrt_(kn * M::inv_u32(Real(0), u2, u)) * xi;
    Real sn, om;
    if (fabs(d) <= Real(1)) {
        const Real r = M::rcp(Real(1) + d * d);
        sn = Real(2) * d * r;
        om = Real(2) * d * d * r;
    } else {
        const Real e = M::rcp(d);
        const Real r = M::rcp(Real(1) + e * e);
        sn = Real(2) * e * r;
        om = Real(2) * r;
    }
    Real sp, cp;
    M::sincos2pi(unif<Real>(wphi), &sp, &cp);
    const Real up2 = g0 * g0 + g1 * g1;
    Real dg[3];
    if (up2 > Real(0)) {
        const Real up = M::sqrt_(up2), rp = M::rcp(up);
        const Real ex = g0 * rp, ey = g1 * rp;
        const Real a = g2 * sn * cp, b = u * sn * sp;
        dg[0] = ex * a - ey * b - g0 * om;
        dg[1] = ey * a + ex * b - g1 * om;
        dg[2] = -up * sn * cp - g2 * om;
    } else {
        dg[0] = u * sn * cp;
        dg[1] = u * sn * sp;
        dg[2] = -g2 * om;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        va[q] += fa * dg[q];
        vb[q] -= fb * dg[q];
    }
}

// Inter-species Coulomb collisions of species pair `pair` in one cell per
// block (Takizuka and Abe for unlike particles), after the intra-species
// pass: the nA particles of the more numerous species (A) each collide once,
// those of the other (B) in turn; collision k joins A pi_A(k) with B
// pi_B(k mod nB) (affine permutations from draw 0 of the cell's stream 5
// with species field 3 + pair) with the random numbers of draw 1 + k/2.
// Thread t follows the B particles r = t, t + T, ...: particle pi_B(r) meets
// A pi_A(r), pi_A(r + nB), ... in that order, its velocity in registers; the
// A particles are disjoint across threads.  A is staged in shared memory
// when it has at most `cap` particles.
template <typename Real>
__global__ void __launch_bounds__(COUL_THREADS, 2)
k_coulomb_inter(WsPtrs W, Pools<Real> P, int par, int pair, int cap)
{
    pdl_wait();
    extern __shared__ __align__(16) unsigned char coul_smem[];
    __shared__ unsigned prm[4];  // a, b of A's permutation, a, b of B's
    const int gw = blockIdx.x;
    const int d = W.cell_disc[gw];
    const Disc &Dd = W.disc[d];
    const int N = Dd.N, c = gw - Dd.ccell_base;
    const int s0 = pair == 2 ? 1 : 0, s1 = pair == 0 ? 1 : 2;
    const int *cs = W.cell_start + Dd.cs_base;
    const int q0 = cs[s0 * (N + 2) + c], n0 = cs[s0 * (N + 2) + c + 1] - q0;
    const int q1 = cs[s1 * (N + 2) + c], n1 = cs[s1 * (N + 2) + c + 1] - q1;
    if (n0 <= 0 || n1 <= 0) return;
    const bool zeroA = n0 >= n1;
    const int sA = zeroA ? s0 : s1, sB = zeroA ? s1 : s0;
    const int nA = zeroA ? n0 : n1, nB = zeroA ? n1 : n0;
    const int pA = zeroA ? q0 : q1, pB = zeroA ? q1 : q0;
    if (nA >= (1 << 29)) {
        if (threadIdx.x == 0) set_status(W.ctl, ST_BADSTATE);
        return;
    }
    if (threadIdx.x == 0) atomicAdd(&W.counters[(size_t)d * C_NCOUNT + C_COUL], (unsigned long long)(nA + nB));
    const unsigned long long step = W.ctl->step[par];
    const unsigned long long seed = Dd.seed;
    const int disc = Dd.discharge;
    const int cur = W.ctl->cur;
    const int sfield = 3 + pair;
    if (threadIdx.x == 0) {
        const uint4 w0 = coulomb_rng(seed, disc, sfield, step, c, 0u);
        const unsigned w[4] = {w0.x, w0.y, w0.z, w0.w};
        const unsigned nn[2] = {(unsigned)nA, (unsigned)nB};
        for (int h = 0; h < 2; ++h) {
            const unsigned un = nn[h];
            unsigned a = 1u, b = 0u;
            if (un >= 2u) {
                a = 1u + w[2 * h] % (un - 1u);
                for (;;) {
                    unsigned x = a, y = un;
                    while (y) {
                        const unsigned t = x % y;
                        x = y;
                        y = t;
                    }
                    if (x == 1u) break;
                    a = a % (un - 1u) + 1u;
                }
                b = w[2 * h + 1] % un;
            }
            prm[2 * h] = a;
            prm[2 * h + 1] = b;
        }
    }
    Real *gax = P.vx[cur] + Dd.pbase[sA] + pA, *gay = P.vy[cur] + Dd.pbase[sA] + pA,
         *gaz = P.vz[cur] + Dd.pbase[sA] + pA;
    Real *gbx = P.vx[cur] + Dd.pbase[sB] + pB, *gby = P.vy[cur] + Dd.pbase[sB] + pB,
         *gbz = P.vz[cur] + Dd.pbase[sB] + pB;
    const bool staged = nA <= cap;
    Real *ax = gax, *ay = gay, *az = gaz;
    if (staged) {
        ax = reinterpret_cast<Real *>(coul_smem);
        ay = ax + cap;
        az = ay + cap;
        coulomb_copy<Real>(ax, ay, az, gax, gay, gaz, nA);
    }
    __syncthreads();
    const unsigned aA = prm[0], bA = prm[1], aB = prm[2], bB = prm[3];
    const unsigned uA = (unsigned)nA, uB = (unsigned)nB;
    const Real kn = pick<Real>(Dd.ci_k[pair], Dd.ci_k_f[pair]) * Real(nB);
    const int ia = zeroA ? 0 : 1;  // index of A's share
    const Real fa = pick<Real>(Dd.ci_frac[pair][ia], Dd.ci_frac_f[pair][ia]);
    const Real fb = pick<Real>(Dd.ci_frac[pair][1 - ia], Dd.ci_frac_f[pair][1 - ia]);
    // indices advanced by additions mod n: j(r) = (aB r + bB) mod nB steps by
    // aB T mod nB, i(k) = (aA k + bA) mod nA by aA T mod nA over r and by
    // aA nB mod nA along a chain
    const unsigned t0 = threadIdx.x;
    unsigned j = (unsigned)(((unsigned long long)aB * t0 + bB) % uB);
    unsigned i0 = (unsigned)(((unsigned long long)aA * t0 + bA) % uA);
    const unsigned stepB = (unsigned)(((unsigned long long)aB * COUL_THREADS) % uB);
    const unsigned stepA = (unsigned)(((unsigned long long)aA * COUL_THREADS) % uA);
    const unsigned chainA = (unsigned)(((unsigned long long)aA * uB) % uA);
    Real m2b = Real(0);  // largest new speed^2 of this thread's B particles
    for (unsigned r = t0; r < uB; r += COUL_THREADS) {
        Real vb[3] = {gbx[j], gby[j], gbz[j]};
        unsigned i = i0;
        for (unsigned k = r; k < uA; k += uB) {
            const uint4 w = coulomb_rng(seed, disc, sfield, step, c, 1u + (k >> 1));
            Real n0r, n1r;
            CoulMath<Real>::normal2(w.x, w.y, n0r, n1r);
            Real va[3] = {ax[i], ay[i], az[i]};
            coulomb_pair_ab<Real>(va, vb, kn, fa, fb, (k & 1u) ? n1r : n0r, (k & 1u) ? w.w : w.z);
            ax[i] = va[0];
            ay[i] = va[1];
            az[i] = va[2];
            i += chainA;
            if (i >= uA) i -= uA;
        }
        gbx[j] = vb[0];
        gby[j] = vb[1];
        gbz[j] = vb[2];
        m2b = fmax(m2b, Real(vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]));
        j += stepB;
        if (j >= uB) j -= uB;
        i0 += stepA;
        if (i0 >= uA) i0 -= uA;
    }
    __syncthreads();
    if (staged) coulomb_copy<Real>(gax, gay, gaz, ax, ay, az, nA);
    // the new speeds raise both species' recorded largest speeds
    vmax_raise(W.vmax2, d * NSP + sA, speed2_max<Real>(ax, ay, az, nA));
    vmax_raise(W.vmax2, d * NSP + sB, (double)m2b);
}

// Births of (19) appended to the electron array of each discharge in cell
// order (the order of the sequential pass).
template <typename Real>
__global__ void __launch_bounds__(256)
k_pair_append(WsPtrs W, Pools<Real> P)
{
    pdl_wait();
    extern __shared__ __align__(16) int pre[];
    __shared__ int wsum[32];
    const int d = blockIdx.x;
    const Disc &Dd = W.disc[d];
    const int N = Dd.N;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        pre[c] = W.pair_bcount[Dd.ccell_base + c];
#pragma unroll
        for (int q = 0; q < NSP; ++q) W.pair_kills[(size_t)(Dd.ccell_base + c) * NSP + q] = 0;
    }
    __syncthreads();
    const int tot = block_scan_exclusive_int(pre, N, wsum);
    if (tot == 0) return;
    const int cur = W.ctl->cur;
    Counts &C = W.cnt[d * NSP + 0];
    const int n0 = C.n;
    typename AccK<Real>::T *acc = AccK<Real>::ptr(W) + Dd.gbase;  // species 0 block
    const PairBirth<Real> *births = reinterpret_cast<const PairBirth<Real> *>(W.pair_births);
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
        const int nbc = W.pair_bcount[Dd.ccell_base + c];
        for (int r = 0; r < nbc; ++r) {
            const PairBirth<Real> &b = births[(size_t)(Dd.ccell_base + c) * PAIR_BIRTH_CAP + r];
            const int dst = n0 + pre[c] + r;
            if (dst >= Dd.cap[0]) {
                set_status(W.ctl, ST_CAPACITY);
                continue;
            }
            const int gidx = Dd.pbase[0] + dst;
            P.cell[cur][gidx] = b.c;
            P.off[cur][gidx] = b.off;
            P.vx[cur][gidx] = b.vx;
            P.vy[cur][gidx] = b.vy;
            P.vz[cur][gidx] = b.vz;
            dep_global(acc, b.c, b.off, 1);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < N; c += blockDim.x) W.pair_bcount[Dd.ccell_base + c] = 0;
    if (threadIdx.x == 0) C.n = min(n0 + tot, Dd.cap[0]);
}

// ------------------------------------------------------------ load / deposit

// Uniform positions in (0, L) and Maxwellian velocities from Philox stream 3
// (step 0, index = slot): draw 0 gives two Box-Muller pairs, draw 1 the
// position.  Computed in FP64 and rounded once to the storage precision.
template <typename Real>
__global__ void k_load(WsPtrs W, Pools<Real> P, const long long *n_init, const double *vt)
{
    const int ds = blockIdx.y;
    const int d = ds / NSP, s = ds % NSP;
    const Disc &Dd = W.disc[d];
    const int n = (int)n_init[ds];
    const int cur = W.ctl->cur;
    const double to_n = Dd.dt / Dd.dx;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 a = rng_block(Dd.seed, Dd.discharge, s, 3, 0, 0, 0ull, (unsigned)i);
        const uint4 b = rng_block(Dd.seed, Dd.discharge, s, 3, 0, 1, 0ull, (unsigned)i);
        double n0, n1, n2, n3;
        box_muller<double>(a.x, a.y, n0, n1);
        box_muller<double>(a.z, a.w, n2, n3);
        const double x = unif<double>(b.x) * Dd.L;
        const double xx = x / Dd.dx;
        int c = (int)floor(xx);
        if (c > Dd.N - 1) c = Dd.N - 1;
        if (c < 0) c = 0;
        Real off = (Real)(xx - c);
        if (off >= Real(1)) {
            if (c + 1 < Dd.N) {
                ++c;
                off = Real(0);
            } else {
                off = Real(0.99999994);
            }
        }
        const int g = Dd.pbase[s] + i;
        P.cell[cur][g] = c;
        P.off[cur][g] = off;
        P.vx[cur][g] = (Real)(vt[ds] * n0 * to_n);
        P.vy[cur][g] = (Real)(vt[ds] * n1 * to_n);
        P.vz[cur][g] = (Real)(vt[ds] * n2 * to_n);
    }
}

// Deposit of every live slot (set-up and after a state change); the caller
// has cleared the accumulators of the affected discharges.
template <typename Real>
__global__ void k_deposit_all(WsPtrs W, Pools<Real> P, int only_disc)
{
    const int ds = blockIdx.y;
    const int d = ds / NSP, s = ds % NSP;
    if (only_disc >= 0 && d != only_disc) return;
    const Disc &Dd = W.disc[d];
    const int n = W.cnt[ds].n;
    const int cur = W.ctl->cur;
    typename AccK<Real>::T *acc = AccK<Real>::ptr(W) + (size_t)s * W.total_nodes + Dd.gbase;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = Dd.pbase[s] + i;
        const int c = P.cell[cur][g];
        if (c >= 0 && c < Dd.N) dep_global(acc, c, P.off[cur][g], 1);
    }
}

// ------------------------------------------------------------ launchers

cudaError_t configure_kernels(bool fp64, LaunchCfg &L)
{
    cudaError_t e;
    L.field_smem = sizeof(double) * (L.maxN + 2) + 16 * (L.maxN + 2) + 16;
    L.sort_smem = sizeof(unsigned short) * SORT_WARPS * ((L.maxN + 2) & ~1);
    L.scatter_smem = sizeof(unsigned short) * SORT_WARPS * ((L.maxN + 2) & ~1);
    if (fp64) {
        e = cudaFuncSetAttribute(k_field<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.field_smem);
        if (e) return e;
        e = cudaFuncSetAttribute(k_sort_count<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.sort_smem);
        if (e) return e;
        e = cudaFuncSetAttribute(k_sort_scatter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.scatter_smem);
        if (e) return e;
        e = cudaFuncSetAttribute(k_coulomb<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)coulomb_smem_bytes(true));
        if (e) return e;
        e = cudaFuncSetAttribute(k_coulomb_inter<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)coulomb_smem_bytes(true));
        if (e) return e;
    } else {
        e = cudaFuncSetAttribute(k_field<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.field_smem);
        if (e) return e;
        e = cudaFuncSetAttribute(k_sort_count<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.sort_smem);
        if (e) return e;
        e = cudaFuncSetAttribute(k_sort_scatter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.scatter_smem);
        if (e) return e;
        e = cudaFuncSetAttribute(k_coulomb<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)coulomb_smem_bytes(false));
        if (e) return e;
        e = cudaFuncSetAttribute(k_coulomb_inter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)coulomb_smem_bytes(false));
        if (e) return e;
    }
    return cudaFuncSetAttribute(k_sort_cellscan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(int) * (L.maxN + 2)));
}

cudaError_t launch_field(bool fp64, bool diag, int mode, const WsPtrs &W, int par, const LaunchCfg &L,
                         cudaStream_t st)
{
    if (fp64)
        launch_k(k_field<double>, W.D, FIELD_THREADS, L.field_smem, st, W, par, diag ? 1 : 0, mode);
    else
        launch_k(k_field<float>, W.D, FIELD_THREADS, L.field_smem, st, W, par, diag ? 1 : 0, mode);
    return cudaGetLastError();
}

int kernels_per_sort() { return 5; }
int kernels_per_pair() { return 7; }

cudaError_t launch_sort(bool fp64, const WsPtrs &W, const void *pools, const int *tab, const LaunchCfg &L,
                        cudaStream_t st)
{
    const size_t scan_smem = sizeof(int) * (L.maxN + 2);
    const int cs_blocks = (L.sort_col_warps * 32 + 255) / 256;
    if (fp64) {
        const Pools<double> &P = *static_cast<const Pools<double> *>(pools);
        launch_k(k_sort_count<double>, L.sort_blocks, SORT_WARPS * 32, L.sort_smem, st, W, P, tab);
        launch_k(k_sort_colscan, cs_blocks, 256, 0, st, W, L.sort_warp_base);
        launch_k(k_sort_cellscan, W.D * NSP, 512, scan_smem, st, W);
        launch_k(k_sort_scatter<double>, L.sort_blocks, SORT_WARPS * 32, L.scatter_smem, st, W, P, tab);
    } else {
        const Pools<float> &P = *static_cast<const Pools<float> *>(pools);
        launch_k(k_sort_count<float>, L.sort_blocks, SORT_WARPS * 32, L.sort_smem, st, W, P, tab);
        launch_k(k_sort_colscan, cs_blocks, 256, 0, st, W, L.sort_warp_base);
        launch_k(k_sort_cellscan, W.D * NSP, 512, scan_smem, st, W);
        launch_k(k_sort_scatter<float>, L.sort_blocks, SORT_WARPS * 32, L.scatter_smem, st, W, P, tab);
    }
    launch_k(k_sort_finish, 1, 256, 0, st, W);
    return cudaGetLastError();
}

size_t coulomb_smem_bytes(bool fp64) { return (size_t)COUL_STAGE * 3 * (fp64 ? 8 : 4); }

cudaError_t launch_coulomb(bool fp64, const WsPtrs &W, const void *pools, int par, cudaStream_t st)
{
    const int grid = W.total_cells * NSP;
    const size_t smem = coulomb_smem_bytes(fp64);
    if (fp64)
        launch_k(k_coulomb<double>, grid, COUL_THREADS, smem, st, W, *static_cast<const Pools<double> *>(pools),
                 par, COUL_STAGE);
    else
        launch_k(k_coulomb<float>, grid, COUL_THREADS, smem, st, W, *static_cast<const Pools<float> *>(pools),
                 par, COUL_STAGE);
    return cudaGetLastError();
}


cudaError_t launch_coulomb_inter(bool fp64, const WsPtrs &W, const void *pools, int par, int pair, cudaStream_t st)
{
    const size_t smem = coulomb_smem_bytes(fp64);
    if (fp64)
        launch_k(k_coulomb_inter<double>, W.total_cells, COUL_THREADS, smem, st, W,
                 *static_cast<const Pools<double> *>(pools), par, pair, COUL_STAGE);
    else
        launch_k(k_coulomb_inter<float>, W.total_cells, COUL_THREADS, smem, st, W,
                 *static_cast<const Pools<float> *>(pools), par, pair, COUL_STAGE);
    return cudaGetLastError();
}

cudaError_t launch_pair_reaction(bool fp64, const WsPtrs &W, const void *pools, int par, int k, cudaStream_t st)
{
    const int fix_blocks = (W.total_cells * 32 + 255) / 256;
    const int eval_blocks = (W.total_cells + 255) / 256;
    if (fp64) {
        const Pools<double> &P = *static_cast<const Pools<double> *>(pools);
        launch_k(k_pair_eval<double>, eval_blocks, 256, 0, st, W, P, par, k);
        launch_k(k_pair_fix<double>, fix_blocks, 256, 0, st, W, P, par, k);
    } else {
        const Pools<float> &P = *static_cast<const Pools<float> *>(pools);
        launch_k(k_pair_eval<float>, eval_blocks, 256, 0, st, W, P, par, k);
        launch_k(k_pair_fix<float>, fix_blocks, 256, 0, st, W, P, par, k);
    }
    return cudaGetLastError();
}

cudaError_t launch_pair_append(bool fp64, const WsPtrs &W, const void *pools, const LaunchCfg &L, cudaStream_t st)
{
    if (fp64)
        launch_k(k_pair_append<double>, W.D, 256, sizeof(int) * (L.maxN + 1), st, W,
                 *static_cast<const Pools<double> *>(pools));
    else
        launch_k(k_pair_append<float>, W.D, 256, sizeof(int) * (L.maxN + 1), st, W,
                 *static_cast<const Pools<float> *>(pools));
    return cudaGetLastError();
}

cudaError_t launch_pair(bool fp64, const WsPtrs &W, const void *pools, int par, const LaunchCfg &L,
                        cudaStream_t st)
{
    for (int k = 0; k < 3; ++k) {
        const cudaError_t e = launch_pair_reaction(fp64, W, pools, par, k, st);
        if (e) return e;
    }
    return launch_pair_append(fp64, W, pools, L, st);
}

cudaError_t launch_retile(const WsPtrs &W, int par, cudaStream_t st)
{
    launch_k(k_retile, 1, 256, 0, st, W, par);
    return cudaGetLastError();
}

cudaError_t launch_load(bool fp64, const WsPtrs &W, const void *pools, const long long *d_ninit,
                        const double *d_vt, int max_n, cudaStream_t st)
{
    dim3 grid((max_n + 255) / 256 > 0 ? ((max_n + 255) / 256 < 4096 ? (max_n + 255) / 256 : 4096) : 1,
              W.D * NSP);
    if (fp64)
        k_load<double><<<grid, 256, 0, st>>>(W, *static_cast<const Pools<double> *>(pools), d_ninit, d_vt);
    else
        k_load<float><<<grid, 256, 0, st>>>(W, *static_cast<const Pools<float> *>(pools), d_ninit, d_vt);
    return cudaGetLastError();
}

cudaError_t launch_deposit_all(bool fp64, const WsPtrs &W, const void *pools, int disc, int max_n,
                               cudaStream_t st)
{
    dim3 grid((max_n + 255) / 256 > 0 ? ((max_n + 255) / 256 < 4096 ? (max_n + 255) / 256 : 4096) : 1,
              W.D * NSP);
    if (fp64)
        k_deposit_all<double><<<grid, 256, 0, st>>>(W, *static_cast<const Pools<double> *>(pools), disc);
    else
        k_deposit_all<float><<<grid, 256, 0, st>>>(W, *static_cast<const Pools<float> *>(pools), disc);
    return cudaGetLastError();
}

} // namespace o2
