// o2pic_host.cu -- the C ABI of libo2pic (declared in include/o2pic.h):
// validation, device constants, workspace carving, the step schedule (CUDA
// graph replay of whole periods), state and diagnostics copies.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/o2pic.h"
#include "o2pic_launch.h"

using namespace o2;

namespace {

constexpr double QE = 1.602176634e-19;
constexpr double ME = 9.1093837015e-31;
constexpr double AMU = 1.66053906660e-27;
constexpr double KB = 1.380649e-23;
constexpr double PI = 3.14159265358979323846;
constexpr double EPS0 = 8.8541878128e-12;
constexpr double M_O = 16.0 * AMU;
constexpr double M_O2 = 32.0 * AMU;
// largest gas-molecule speed a collision can draw, in thermal speeds
// sqrt(kT/M_O2): two Box-Muller pairs of radius at most sqrt(66 ln 2) = 6.77
// (the smallest FP64 uniform is 2^-33; FP32 2^-24), so at most 9.58
constexpr double GAS_SPEED_MAX = 10.0;
// O- carries the extra electron and O2+ lacks one, so that every reaction of
// Table I conserves mass exactly.
const double MASS[3] = {ME, M_O + ME, M_O2 - ME};
const double CHARGE[3] = {-QE, -QE, QE};

thread_local std::string g_err;

int proj_of(int r)
{
    switch (r) {
    case 5: case 14: case 16: case 17: return 1;
    case 6: return 2;
    default: return 0;
    }
}
int targ_of(int r)
{
    if (r == 13 || r == 14) return 2;
    if (r == 19) return 1;
    return -1;
}

struct HostTable {
    int reaction, sub, n;
    std::vector<double> E, S;
    double th;
};

// sigma(E): linear between nodes, end values held, zero below threshold
double sigma_host(const HostTable &t, double E)
{
    if (E < t.th) return 0.0;
    if (E <= t.E[0]) return t.S[0];
    if (E >= t.E[t.n - 1]) return t.S[t.n - 1];
    int k = int(std::upper_bound(t.E.begin(), t.E.end(), E) - t.E.begin()) - 1;
    k = std::max(0, std::min(k, t.n - 2));
    double f = (E - t.E[k]) / (t.E[k + 1] - t.E[k]);
    return t.S[k] + f * (t.S[k + 1] - t.S[k]);
}

struct Bump {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = (off + 255) & ~size_t(255);
        off = o + bytes;
        return o;
    }
};

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    size_t colscan_agg, sort_whist, ctl, disc, cnt, phi_s2_sum, phi0_sum, D0_sum, gtab, gtabf, gpm, gpmf, tile_cnt, births, births_lb, sort_tot, warp_base, pair_first, vmax2, nubin, cand, pair_kills, pair_tab[3], acc, Efield, Ereal, phi, rho, dens, dens_sum, phi_sum, nsamp,
        counters, eedf, iedf, fm, tables, lutE, lutS, lutEf, lutSf, sort_counts, cell_start,
        sort_live, pair_bcount, cell_disc, pair_births, sort_tab, ninit, vt;
    size_t cell[2], off[2], vx[2], vy[2], vz[2];
    size_t total;
    int total_nodes, total_cells, max_chunks, total_cap, sort_blocks, n_lut, maxN, eedf_max, fm_max, cand_cap;
    int birth_cap;
    long long colscan_units;  // warps of the sort's column scan
    long long gtab_n;  // elements of the node-major gas tables
    std::vector<int> pbase, capr, gbase, ccell, sort_cbase, sort_gmax, cs_base, eedf_base, iedf_base,
        fm_base;
};

bool validate(const pic_config *c, int D, const pic_xs_table *xs, int n_xs, std::string &why)
{
    if (!c || D < 1 || D > MAX_DISCHARGES) {
        why = "n_discharges must be in [1, 1024]";
        return false;
    }
    for (int d = 0; d < D; ++d) {
        const pic_config &q = c[d];
        char b[256];
        if (!(q.L_m > 0) || !(q.dt_s > 0) || q.n_cells < 2 || q.n_cells > 4096 || !(q.weight_m2 >= 0) ||
            !(q.p_Pa >= 0) || !(q.T_gas_K > 0) || !(q.numax_safety >= 1.0) || q.numax_bins < 0 ||
            q.numax_bins > NUBIN_MAX) {
            snprintf(b, sizeof b, "discharge %d: need L > 0, dt > 0, 2 <= n_cells <= 4096, weight >= 0, "
                                  "p >= 0, T > 0, numax_safety >= 1, 0 <= numax_bins <= 64", d);
            why = b;
            return false;
        }
        if (q.precision != c[0].precision || q.diag_every != c[0].diag_every || q.n1 != c[0].n1 ||
            q.sort_interval != c[0].sort_interval || q.n2 != c[0].n2) {
            why = "all discharges of one handle must share precision, diag_every, n1, n2 and sort_interval";
            return false;
        }
        if (q.n2 < 0 || (q.n2 > 0 && !(q.coulomb_log > 0))) {
            why = "n2 must be >= 0 and coulomb_log > 0 when n2 > 0";
            return false;
        }
        if (q.gas_scheme != 0 && q.gas_scheme != 1) {
            why = "gas_scheme must be 0 (null collision) or 1 (sequential list)";
            return false;
        }
        if (q.gas_scheme == 1 && q.n1 <= 0) {
            why = "the sequential gas scheme (gas_scheme = 1) needs n1 > 0";
            return false;
        }
        if (q.ion_subcycle < 0 || (q.ion_subcycle > 1 && q.diag_every > 0 && q.diag_every % q.ion_subcycle != 0)) {
            why = "ion_subcycle must be >= 0, and diag_every a multiple of it";
            return false;
        }
        if (q.coulomb_inter != 0 && q.coulomb_inter != 1) {
            why = "coulomb_inter must be 0 or 1";
            return false;
        }
        if (q.gas_scheme != c[0].gas_scheme || q.coulomb_inter != c[0].coulomb_inter) {
            why = "all discharges of one handle must share gas_scheme and coulomb_inter";
            return false;
        }
        if (q.precision != PIC_FP64 && q.precision != PIC_FP32_MIXED) {
            why = "precision must be PIC_FP64 or PIC_FP32_MIXED";
            return false;
        }
        if (q.n1 < 0 || q.sort_interval < 0 || q.diag_every < 0) {
            why = "n1, sort_interval and diag_every must be >= 0";
            return false;
        }
        if (q.eedf_bins < 0 || q.iedf_bins < 0 || q.fm_bins < 0 || q.eedf_bins > 4096 ||
            q.iedf_bins > 4096 || (q.fm_bins > 0 && (q.fm_xbins < 1 || q.fm_xbins * q.fm_bins > 16384))) {
            why = "histogram sizes out of range (eedf, iedf <= 4096; fm_xbins*fm_bins <= 16384)";
            return false;
        }
        if ((q.eedf_bins > 0 && !(q.eedf_emax_eV > 0)) || (q.iedf_bins > 0 && !(q.iedf_emax_eV > 0)) ||
            (q.fm_bins > 0 && !(q.fm_emax_eV > 0))) {
            why = "histogram ranges must be > 0";
            return false;
        }
        for (int s = 0; s < 3; ++s) {
            if (q.n_init[s] < 0 || q.capacity[s] < q.n_init[s] || q.capacity[s] > (1LL << 30) ||
                !(q.T0_eV[s] >= 0) || !(q.ecap_eV[s] > 0)) {
                snprintf(b, sizeof b, "discharge %d species %d: need 0 <= n_init <= capacity <= 2^30, "
                                      "T0 >= 0, ecap > 0", d, s);
                why = b;
                return false;
            }
        }
    }
    {
        // slot indices are int and the births' tags carry the tile index in
        // 21 bits: all slots, with the alignment padding, below 2^31
        long long slots = 0;
        for (int d = 0; d < D; ++d) {
            for (int s = 0; s < 3; ++s)
                slots += ((std::max(1LL, c[d].capacity[s]) + CHUNK - 1) / CHUNK) * (long long)CHUNK;
            slots += (long long)(TILE_ALIGN + 3 * TILES_PER_TICKET) * CHUNK;
        }
        if (slots >= (1LL << 31)) {
            why = "the capacities of all discharges together must stay below 2^31 slots";
            return false;
        }
    }
    if (n_xs < 0 || (n_xs > 0 && !xs)) {
        why = "bad table list";
        return false;
    }
    int ngas[3] = {0, 0, 0}, npair[20] = {0};
    int first[3] = {-1, -1, -1};
    for (int i = 0; i < n_xs; ++i) {
        const pic_xs_table &t = xs[i];
        char b[256];
        if (t.reaction < 4 || t.reaction > 19 || t.n < 2 || !t.E_eV || !t.sigma_m2 || !(t.threshold_eV >= 0)) {
            snprintf(b, sizeof b, "table %d: reaction must be 4..19, n >= 2, threshold >= 0", i);
            why = b;
            return false;
        }
        if (!(t.E_eV[0] > 0)) {
            snprintf(b, sizeof b, "table %d: first node must be > 0", i);
            why = b;
            return false;
        }
        for (int k = 0; k + 1 < t.n; ++k)
            if (!(t.E_eV[k + 1] > t.E_eV[k])) {
                snprintf(b, sizeof b, "table %d: nodes must increase strictly", i);
                why = b;
                return false;
            }
        // geometric grid (the device locates the segment by a logarithm)
        const double r = std::log(t.E_eV[t.n - 1] / t.E_eV[0]) / (t.n - 1);
        for (int k = 0; k < t.n; ++k)
            if (std::fabs(std::log(t.E_eV[k] / t.E_eV[0]) - k * r) > 0.25 * r) {
                snprintf(b, sizeof b, "table %d: nodes must be geometric", i);
                why = b;
                return false;
            }
        if (targ_of(t.reaction) >= 0) {
            if (++npair[t.reaction] > 1) {
                why = "at most one table per particle-target reaction";
                return false;
            }
        } else {
            const int s = proj_of(t.reaction);
            if (++ngas[s] > MAX_GAS_CH) {
                why = "too many gas channels for one projectile (max 16)";
                return false;
            }
            if (first[s] < 0) {
                first[s] = i;
            } else {
                const pic_xs_table &f = xs[first[s]];
                bool same = f.n == t.n;
                for (int k = 0; same && k < t.n; ++k)
                    same = std::fabs(f.E_eV[k] - t.E_eV[k]) <= 1e-12 * f.E_eV[k];
                if (!same) {
                    snprintf(b, sizeof b, "table %d: gas channels of one projectile must share one grid", i);
                    why = b;
                    return false;
                }
            }
        }
    }
    return true;
}

Layout make_layout(const pic_config *c, int D, const pic_xs_table *xs, int n_xs, bool fp64)
{
    Layout L{};
    const size_t R = fp64 ? 8 : 4;
    int tn = 0, tc = 0, mc = 0, cap = 0, sb = 0, maxN = 0, em = 0, fmm = 0;
    long long sortc = 0, csb = 0, eb = 0, ib = 0, fb = 0;
    L.pbase.resize(3 * D);
    L.capr.resize(3 * D);
    L.sort_cbase.resize(3 * D);
    L.sort_gmax.resize(3 * D);
    for (int d = 0; d < D; ++d) {
        const int N = c[d].n_cells;
        mc = (mc + TILE_ALIGN - 1) / TILE_ALIGN * TILE_ALIGN;  // tiles of a discharge start aligned
        L.gbase.push_back(tn);
        L.ccell.push_back(tc);
        L.cs_base.push_back((int)csb);
        L.eedf_base.push_back((int)eb);
        L.iedf_base.push_back((int)ib);
        L.fm_base.push_back((int)fb);
        tn += N + 1;
        tc += N;
        csb += 3LL * (N + 2);
        eb += c[d].eedf_bins;
        ib += 2LL * c[d].iedf_bins;
        fb += (long long)c[d].fm_xbins * c[d].fm_bins;
        maxN = std::max(maxN, N);
        em = std::max(em, c[d].eedf_bins);
        fmm = std::max(fmm, c[d].fm_xbins * c[d].fm_bins);
        for (int s = 0; s < 3; ++s) {
            const int cr = (int)round_up((size_t)std::max(1LL, c[d].capacity[s]), CHUNK);
            L.pbase[3 * d + s] = cap;
            L.capr[3 * d + s] = cr;
            cap += cr;
            mc = (mc + TILES_PER_TICKET - 1) / TILES_PER_TICKET * TILES_PER_TICKET;
            mc += cr / CHUNK;
            const int g = (cr + SORT_CHUNK - 1) / SORT_CHUNK;
            L.sort_gmax[3 * d + s] = g;
            L.colscan_units += (long long)((N + 1 + 31) / 32) * ((g + COLSCAN_SEG - 1) / COLSCAN_SEG);
            L.sort_cbase[3 * d + s] = (int)sortc;
            sortc += (long long)g * (N + 1);
            sb += g;
        }
    }
    mc = (mc + TILE_ALIGN - 1) / TILE_ALIGN * TILE_ALIGN;  // room for the padding after the last species
    int nl = 0;
    for (int i = 0; i < n_xs; ++i) nl += xs[i].n;
    // node-major gas tables: per (d, s), rows of the shared grid, 4-padded
    long long gn = 0;
    {
        int nodes[3] = {0, 0, 0}, nch[3] = {0, 0, 0};
        for (int i = 0; i < n_xs; ++i) {
            if (targ_of(xs[i].reaction) >= 0) continue;
            const int s = proj_of(xs[i].reaction);
            nodes[s] = xs[i].n;
            ++nch[s];
        }
        for (int s = 0; s < 3; ++s) gn += (long long)nodes[s] * ((nch[s] + 3) / 4 * 4) + 4;
        gn *= D;
    }
    L.gtab_n = gn;
    L.total_nodes = tn;
    L.total_cells = tc;
    L.max_chunks = mc;
    L.total_cap = cap;
    L.sort_blocks = sb;
    L.n_lut = nl;
    L.maxN = maxN;
    L.eedf_max = em;
    L.fm_max = fmm;
    Bump B;
    L.ctl = B.take(sizeof(Ctl));
    L.disc = B.take(sizeof(Disc) * D);
    L.cnt = B.take(sizeof(Counts) * 3 * D);
    L.tile_cnt = B.take(4ull * 3 * SUBTILES * mc);
    L.birth_cap = c[0].gas_scheme == 1 ? BIRTH_CAP_SEQ : BIRTH_CAP_W;
    L.births = B.take((size_t)mc * SUBTILES * L.birth_cap * (fp64 ? 40 : 24));
    L.births_lb = B.take(8ull * 3 * (mc / TILE_ALIGN + 1));
    L.acc = B.take(8ull * 3 * tn);
    L.Efield = B.take(8ull * tn);
    L.Ereal = B.take(R * tn);
    L.phi = B.take(8ull * tn);
    L.rho = B.take(8ull * tn);
    L.dens = B.take(8ull * 3 * tn);
    L.dens_sum = B.take(8ull * 3 * tn);
    L.phi_sum = B.take(8ull * tn);
    L.nsamp = B.take(8ull * D);
    L.phi_s2_sum = B.take(16ull * tn);
    L.phi0_sum = B.take(8ull * D);
    L.D0_sum = B.take(8ull * D);
    L.counters = B.take(8ull * C_NCOUNT * D);
    L.eedf = B.take(4ull * std::max(1LL, eb));
    L.iedf = B.take(4ull * std::max(1LL, ib));
    L.fm = B.take(4ull * std::max(1LL, fb));
    L.tables = B.take(sizeof(TableDesc) * std::max(1, n_xs));
    L.lutE = B.take(8ull * std::max(1, nl));
    L.lutS = B.take(8ull * std::max(1, nl));
    L.lutEf = B.take(4ull * std::max(1, nl));
    L.lutSf = B.take(4ull * std::max(1, nl));
    L.gtab = B.take(8ull * std::max(1LL, gn));
    L.gtabf = B.take(4ull * std::max(1LL, gn));
    L.gpm = B.take(8ull * std::max(1LL, gn));
    L.gpmf = B.take(4ull * std::max(1LL, gn));
    L.sort_counts = B.take(4ull * std::max(1LL, sortc));
    L.sort_whist = B.take(2ull * SORT_WARPS * std::max(1LL, sortc));
    L.cell_start = B.take(4ull * csb);
    L.sort_live = B.take(4ull * 3 * D);
    L.sort_tot = B.take(4ull * csb);
    L.warp_base = B.take(4ull * (3 * D + 1));
    L.colscan_agg = B.take(8ull * 32 * (size_t)std::max(1LL, L.colscan_units));
    L.pair_bcount = B.take(4ull * tc);
    L.cell_disc = B.take(4ull * tc);
    L.pair_first = B.take(4ull * tc);
    L.vmax2 = B.take(8ull * 3 * D);
    L.nubin = B.take(sizeof(NuBin) * NUBIN_MAX * (size_t)D);
    // collision candidates of one step: a quarter of all slots (a candidate
    // probability up to 1/4 on average); more is reported as PIC_ECAPACITY
    L.cand_cap = (int)std::min<long long>((long long)cap / 4 + 65536, (1LL << 31) - 1);
    L.cand = B.take(8ull * (size_t)L.cand_cap);
    L.pair_kills = B.take(4ull * 3 * tc);
    for (int s = 0; s < 3; ++s) {
        long long tiles = 0;
        for (int d = 0; d < D; ++d) tiles += (c[d].capacity[s] + 255) / 256;
        L.pair_tab[s] = B.take(8ull * std::max(1LL, tiles));
    }
    L.pair_births = B.take((size_t)tc * PAIR_BIRTH_CAP * (8 + 4 * 8));
    L.sort_tab = B.take(8ull * sb);
    L.ninit = B.take(8ull * 3 * D);
    L.vt = B.take(8ull * 3 * D);
    for (int b = 0; b < 2; ++b) {
        L.cell[b] = B.take(4ull * cap);
        L.off[b] = B.take(R * cap);
        L.vx[b] = B.take(R * cap);
        L.vy[b] = B.take(R * cap);
        L.vz[b] = B.take(R * cap);
    }
    L.total = round_up(B.off, 256);
    return L;
}

} // namespace

struct pic_handle {
    int D = 0;
    bool fp64 = false;
    std::vector<pic_config> cfg;
    std::vector<HostTable> tabs;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    Layout lay;
    WsPtrs W{};
    Pools<float> Pf{};
    Pools<double> Pd{};
    LaunchCfg L{};
    int *sort_tab = nullptr;
    long long step = 0;
    std::vector<Disc> disc;
    std::vector<NuBin> nubin;   // [D * NUBIN_MAX]
    std::vector<double> numax;  // [D*3]
    std::string err;
    // largest accepted fraction of nu_max violations among null-collision
    // candidates and of Eq. 1 P > 1 clamps among Eq. 1 evaluations
    double numeric_budget = 1e-6;
    // captured graphs: one RF cycle (the whole cycle's kernels; cycle_steps
    // time steps, a multiple of the schedule's period) and one period of the
    // step schedule (for what is left of a call)
    cudaGraphExec_t gexec = nullptr;        // one period
    cudaGraphExec_t gexec_cycle = nullptr;  // one RF cycle
    long long period = 0;
    long long cycle_steps = 0;              // 0: the cycle is not captured
    long long graph_launches = 0;           // kernels in the period graph
    long long cycle_graph_launches = 0;     // kernels in the cycle graph
    long long graph_calls = 0;              // cudaGraphLaunch calls since pic_init
    bool graph_failed = false;
    // timing
    bool timing = false;
    // device ms and timed launches per kernel kind (push, Coulomb, sequential
    // gas, push with diagnostics)
    double kms[4] = {0.0, 0.0, 0.0, 0.0};
    long long kl[4] = {0, 0, 0, 0};
    long long launches = 0;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;          // kind of each event pair
    int ev_used = 0;
    unsigned long long slots0 = 0, cands0 = 0, bslots0 = 0, bcands0 = 0, coul0 = 0, dsmc0 = 0;
    const void *pools() const { return fp64 ? (const void *)&Pd : (const void *)&Pf; }
};

static pic_status fail(pic_handle *h, pic_status s, const std::string &m)
{
    if (h) h->err = m;
    g_err = m;
    return s;
}

static pic_status cuda_fail(pic_handle *h, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, PIC_ECUDA, m);
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);     \
    } while (0)

extern "C" size_t pic_workspace_size(const pic_config *cfgs, int n_discharges, const pic_xs_table *xs, int n_xs)
{
    std::string why;
    if (!validate(cfgs, n_discharges, xs, n_xs, why)) {
        g_err = why;
        return 0;
    }
    return make_layout(cfgs, n_discharges, xs, n_xs, cfgs[0].precision == PIC_FP64).total;
}

static void build_disc(pic_handle *h, int d, const std::vector<int> &gas_tabs_by_sp_flat,
                       const std::vector<int> &gas_count, const int pair_tab[20])
{
    const pic_config &q = h->cfg[d];
    const Layout &L = h->lay;
    Disc D{};
    const int N = q.n_cells;
    D.N = N;
    D.gbase = L.gbase[d];
    for (int s = 0; s < 3; ++s) {
        D.pbase[s] = L.pbase[3 * d + s];
        D.cap[s] = (int)q.capacity[s];
        D.sort_cbase[s] = L.sort_cbase[3 * d + s];
        D.sort_gmax[s] = L.sort_gmax[3 * d + s];
    }
    D.ccell_base = L.ccell[d];
    D.cs_base = L.cs_base[d];
    D.dx = q.L_m / N;
    D.dt = q.dt_s;
    D.L = q.L_m;
    D.weight = q.weight_m2;
    D.U_rf = q.U_rf_V;
    D.omega = 2.0 * PI * q.f_rf_Hz;
    D.phase = q.rf_phase;
    const double tdx = q.dt_s / D.dx, xdt = D.dx / q.dt_s;
    D.kE = q.dt_s * q.dt_s / D.dx;
    D.dens_fix = q.weight_m2 / (D.dx * (double)(1 << FIX_BITS));
    D.dens_fix_wall = q.weight_m2 / (0.5 * D.dx * (double)(1 << FIX_BITS));
    D.Kfix = QE * q.weight_m2 / (double)(1 << FIX_BITS) / 8.8541878128e-12;
    const double mu2 = M_O * MASS[1] / (M_O + MASS[1]);
    D.mu2_15 = mu2;
    D.f15 = 2.0 * QE * mu2 / (MASS[1] * MASS[1]) * tdx * tdx;
    D.f16 = std::sqrt(MASS[1] / (10.0 * ME));
    D.f17 = 2.0 * QE / ME * tdx * tdx;
    D.eedf_bins = q.eedf_bins;
    D.iedf_bins = q.iedf_bins;
    D.fm_bins = q.fm_bins;
    D.fm_xbins = q.fm_bins > 0 ? q.fm_xbins : 0;
    D.eedf_scale = q.eedf_bins > 0 ? q.eedf_bins / q.eedf_emax_eV : 0.0;
    D.iedf_scale = q.iedf_bins > 0 ? q.iedf_bins / q.iedf_emax_eV : 0.0;
    D.fm_scale = q.fm_bins > 0 ? q.fm_bins / (2.0 * q.fm_emax_eV) : 0.0;
    D.fm_emax = q.fm_emax_eV;
    D.f15_f = (float)D.f15;
    D.f16_f = (float)D.f16;
    D.f17_f = (float)D.f17;
    D.eedf_scale_f = (float)D.eedf_scale;
    D.iedf_scale_f = (float)D.iedf_scale;
    D.fm_scale_f = (float)D.fm_scale;
    D.fm_emax_f = (float)D.fm_emax;
    D.eedf_base = L.eedf_base[d];
    D.iedf_base = L.iedf_base[d];
    D.fm_base = L.fm_base[d];
    D.diag_every = q.diag_every;
    D.n1 = q.n1;
    D.sort_interval = q.sort_interval;
    D.n2 = q.n2;
    D.seed = q.seed;
    D.discharge = d;
    D.cx_iso = q.cx_isotropic;
    D.gas_scheme = q.gas_scheme;
    D.ion_sub = q.ion_subcycle > 1 ? q.ion_subcycle : 1;
    D.coul_inter = (q.n2 > 0 && q.coulomb_inter) ? 1 : 0;
    {
        const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        const double tdx_ = q.dt_s / D.dx, xdt_ = D.dx / q.dt_s;
        (void)tdx_;
        for (int k = 0; k < 3; ++k) {
            const double ma = MASS[pr[k][0]], mb = MASS[pr[k][1]], mu = ma * mb / (ma + mb);
            const double qq = CHARGE[pr[k][0]] * CHARGE[pr[k][1]];
            D.ci_k[k] = q.n2 > 0 ? qq * qq * q.coulomb_log * (q.n2 * q.dt_s) * q.weight_m2 /
                                       (8.0 * PI * EPS0 * EPS0 * mu * mu * D.dx) / (xdt_ * xdt_ * xdt_)
                                 : 0.0;
            D.ci_frac[k][0] = mb / (ma + mb);
            D.ci_frac[k][1] = ma / (ma + mb);
            D.ci_k_f[k] = (float)D.ci_k[k];
            D.ci_frac_f[k][0] = (float)D.ci_frac[k][0];
            D.ci_frac_f[k][1] = (float)D.ci_frac[k][1];
        }
    }
    const double ngas = q.p_Pa / (KB * q.T_gas_K);
    for (int s = 0; s < 3; ++s) {
        SpeciesC &S = D.sp[s];
        const double m = MASS[s];
        const double mu = m * M_O2 / (m + M_O2);
        S.qm = CHARGE[s] / m * q.dt_s * q.dt_s / D.dx;
        S.vgas_n = std::sqrt(KB * q.T_gas_K / M_O2) * tdx;
        S.Ek = 0.5 * mu * xdt * xdt / QE;
        S.ke_eV = 0.5 * m * xdt * xdt / QE;
        S.mfrac = m / (m + M_O2);
        S.Mfrac = M_O2 / (m + M_O2);
        S.vscale = xdt;
        // Eq. 2 (eps0 squared, reduced mass m/2 of a like pair) with the
        // cell density count * weight / dx and tau = n2 dt, in units of u_n^3
        const double mc = 0.5 * m, q2 = CHARGE[s] * CHARGE[s];
        S.coul_k = q.n2 > 0 ? q2 * q2 * q.coulomb_log * (q.n2 * q.dt_s) * q.weight_m2 /
                                  (8.0 * PI * EPS0 * EPS0 * mc * mc * D.dx) / (xdt * xdt * xdt)
                            : 0.0;
        S.nch = gas_count[s];
        S.table_lo = S.nch > 0 ? gas_tabs_by_sp_flat[s * MAX_GAS_CH] : 0;
        for (int j = 0; j < S.nch; ++j) {
            const int ti = gas_tabs_by_sp_flat[s * MAX_GAS_CH + j];
            const HostTable &t = h->tabs[ti];
            S.ch[j].table = ti;
            S.ch[j].reaction = t.reaction;
            const double nj = (t.reaction == 17) ? q.C_delta * ngas : ngas;
            S.ch[j].coef = nj * D.dx;
            S.ch[j].dloss = 2.0 * t.th * QE / mu * tdx * tdx;
            S.ch[j].coef_f = (float)S.ch[j].coef;
            S.ch[j].dloss_f = (float)S.ch[j].dloss;
            S.ch[j].th = t.th;
            S.ch[j].th_f = (float)t.th;
        }
        // nu_max up to a centre-of-mass energy capE: [0, capE] is cut at every
        // node and threshold of the species' channels; between neighbouring
        // cuts a < b every sigma_j is linear (or zero), so sum_j n_j
        // max(sigma_j(a), sigma_j(b)) sqrt(2b/mu) bounds the frequency there;
        // the largest over the intervals, times the safety factor
        auto numax_upto = [&](double capE) {
            std::vector<double> cut{0.0, capE};
            for (int a = 0; a < S.nch; ++a) {
                const HostTable &ta = h->tabs[S.ch[a].table];
                for (int k = 0; k < ta.n; ++k)
                    if (ta.E[k] > 0.0 && ta.E[k] < capE) cut.push_back(ta.E[k]);
                if (ta.th > 0.0 && ta.th < capE) cut.push_back(ta.th);
            }
            std::sort(cut.begin(), cut.end());
            double best = 0.0;
            for (size_t i = 0; i + 1 < cut.size(); ++i) {
                const double a = cut[i], b = cut[i + 1];
                if (!(b > a)) continue;
                const double u = std::sqrt(2.0 * b * QE / mu);
                double nu = 0.0;
                for (int c = 0; c < S.nch; ++c) {
                    const HostTable &tc = h->tabs[S.ch[c].table];
                    const double nj = (tc.reaction == 17) ? q.C_delta * ngas : ngas;
                    nu += nj * std::max(sigma_host(tc, a), sigma_host(tc, b)) * u;
                }
                best = std::max(best, nu);
            }
            return best * q.numax_safety;
        };
        S.numax = numax_upto(q.ecap_eV[s]);
        // electrons: one bound per quarter octave of lab energy; a bin's
        // relative speed is at most its top electron speed plus the largest
        // gas-molecule speed a collision can draw (Box-Muller radius at the
        // smallest uniform 2^-33: below 9.6 thermal speeds sqrt(kT/M_O2),
        // taken as GAS_SPEED_MAX); the last bin keeps the species' bound
        S.nbins = (s == 0) ? q.numax_bins : 0;
        S.bin_off = d * NUBIN_MAX;
        for (int b = 0; b < S.nbins; ++b) {
            NuBin &nb = h->nubin[(size_t)d * NUBIN_MAX + b];
            double nu = S.numax;
            if (b < S.nbins - 1) {
                const double Ktop = std::ldexp(1.0 + (b % 4 + 1) / 4.0, NUBIN_LOG2_E0 + b / 4);
                const double urel = std::sqrt(2.0 * Ktop * QE / m) + GAS_SPEED_MAX * std::sqrt(KB * q.T_gas_K / M_O2);
                nu = numax_upto(0.5 * mu * urel * urel / QE);
            }
            const double pb = 1.0 - std::exp(-nu * q.dt_s);
            const double tb = std::ceil(pb * 4294967296.0 - 0.5);
            nb.tnull = tb <= 0.0 ? 0u : (tb >= 4294967295.0 ? 0xFFFFFFFFu : (unsigned)tb);
            if (q.gas_scheme == 1) nb.tnull = 0u;  // no null-collision candidates
            nb.numax_n = nu * q.dt_s;
            nb.numax_n_f = (float)nb.numax_n;
        }
        S.numax_n = S.numax * q.dt_s;
        // a sub-cycled ion is tested once per push, over ion_sub steps
        const double pnull = 1.0 - std::exp(-S.numax * q.dt_s * (s > 0 ? D.ion_sub : 1));
        const double thr = std::ceil(pnull * 4294967296.0 - 0.5);
        S.tnull = thr <= 0.0 ? 0u : (thr >= 4294967295.0 ? 0xFFFFFFFFu : (unsigned)thr);
        if (q.gas_scheme == 1) S.tnull = 0u;  // no null-collision candidates
        S.qm_f = (float)S.qm;
        S.numax_n_f = (float)S.numax_n;
        S.vgas_n_f = (float)S.vgas_n;
        S.Ek_f = (float)S.Ek;
        S.mfrac_f = (float)S.mfrac;
        S.Mfrac_f = (float)S.Mfrac;
        S.ke_eV_f = (float)S.ke_eV;
        S.coul_k_f = (float)S.coul_k;
        h->numax[3 * d + s] = S.numax;
    }
    // the sequential scheme's list: gas channels in the order of Table I
    // (reaction number, then table order)
    D.ndsmc = 0;
    for (int r = 4; r <= 18; ++r)
        for (size_t ti = 0; ti < h->tabs.size(); ++ti) {
            if (h->tabs[ti].reaction != r) continue;
            for (int s = 0; s < 3; ++s)
                for (int j = 0; j < D.sp[s].nch; ++j)
                    if (D.sp[s].ch[j].table == (int)ti && D.ndsmc < MAX_DSMC) D.dsmc[D.ndsmc++] = DsmcCh{s, j, r, 0};
        }
    const int rx[3] = {13, 14, 19};
    for (int k = 0; k < 3; ++k) {
        PairC &P = D.pair[k];
        P.table = pair_tab[rx[k]];
        P.proj = proj_of(rx[k]);
        P.targ = targ_of(rx[k]);
        const double mp = MASS[P.proj], mt = MASS[P.targ];
        const double mu = mp * mt / (mp + mt);
        P.coef = q.weight_m2 * q.n1;
        P.Ek = 0.5 * mu * xdt * xdt / QE;
        P.mfrac = mp / (mp + mt);
        P.Mfrac = mt / (mp + mt);
        P.dloss = P.table >= 0 ? 2.0 * h->tabs[P.table].th * QE / mu * tdx * tdx : 0.0;
        P.Ek_f = (float)P.Ek;
        P.mfrac_f = (float)P.mfrac;
        P.Mfrac_f = (float)P.Mfrac;
        P.dloss_f = (float)P.dloss;
        P.coef_f = (float)P.coef;
        // Bound on sigma(E) u over the table, u in cells per step: on a
        // segment [E_k, E_k+1] sigma is at most the larger end value and
        // u <= U_k+1 = sqrt(E_k+1 / Ek); below the grid sigma is the first
        // value and u < U_0; above it sigma is the last value, so sigma u
        // grows as bnd_s * u.  A relative margin covers the rounding of the
        // device's sigma, u and E.
        P.bnd_g = P.bnd_s = 0.0;
        if (P.table >= 0) {
            const HostTable &t = h->tabs[P.table];
            const int n = (int)t.E.size();
            double g = t.S[0] * std::sqrt(t.E[0] / P.Ek);
            for (int q = 0; q + 1 < n; ++q)
                g = std::max(g, std::max(t.S[q], t.S[q + 1]) * std::sqrt(t.E[q + 1] / P.Ek));
            P.bnd_g = g * 1.001;
            P.bnd_s = t.S[n - 1] * 1.001;
        }
        P.bnd_g_f = (float)(P.bnd_g * 1.0001);
        P.bnd_s_f = (float)(P.bnd_s * 1.0001);
    }
    h->disc[d] = D;
}

extern "C" pic_status pic_init(const pic_config *cfgs, int n_discharges, const pic_xs_table *xs, int n_xs,
                               void *d_workspace, size_t ws_bytes, void *cuda_stream, pic_handle **out)
{
    if (!out) return fail(nullptr, PIC_EINVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!validate(cfgs, n_discharges, xs, n_xs, why)) return fail(nullptr, PIC_EINVAL, why);
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255))
        return fail(nullptr, PIC_EINVAL, "workspace must be a 256-byte aligned device pointer");
    pic_handle *h = new pic_handle();
    h->D = n_discharges;
    h->fp64 = cfgs[0].precision == PIC_FP64;
    h->cfg.assign(cfgs, cfgs + n_discharges);
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->lay = make_layout(cfgs, n_discharges, xs, n_xs, h->fp64);
    if (ws_bytes < h->lay.total) {
        delete h;
        return fail(nullptr, PIC_ENOMEM, "workspace smaller than pic_workspace_size()");
    }
    h->ws = static_cast<char *>(d_workspace);
    for (int i = 0; i < n_xs; ++i) {
        HostTable t;
        t.reaction = xs[i].reaction;
        t.sub = xs[i].sub;
        t.n = xs[i].n;
        t.E.assign(xs[i].E_eV, xs[i].E_eV + t.n);
        t.S.assign(xs[i].sigma_m2, xs[i].sigma_m2 + t.n);
        t.th = xs[i].threshold_eV;
        h->tabs.push_back(t);
    }
    const Layout &L = h->lay;
    char *b = h->ws;
    WsPtrs &W = h->W;
    W.ctl = reinterpret_cast<Ctl *>(b + L.ctl);
    W.disc = reinterpret_cast<Disc *>(b + L.disc);
    W.cnt = reinterpret_cast<Counts *>(b + L.cnt);
    W.chunk_ds = nullptr;
    W.tile_cnt = reinterpret_cast<int *>(b + L.tile_cnt);
    W.births = b + L.births;
    W.birth_cap = L.birth_cap;
    W.births_lb = reinterpret_cast<unsigned long long *>(b + L.births_lb);
    W.colscan_agg = reinterpret_cast<unsigned long long *>(b + L.colscan_agg);
    W.acc_fix = reinterpret_cast<unsigned long long *>(b + L.acc);
    W.acc_dbl = reinterpret_cast<double *>(b + L.acc);
    W.Efield = reinterpret_cast<double *>(b + L.Efield);
    W.Ereal = b + L.Ereal;
    W.phi = reinterpret_cast<double *>(b + L.phi);
    W.rho = reinterpret_cast<double *>(b + L.rho);
    W.dens = reinterpret_cast<double *>(b + L.dens);
    W.dens_sum = reinterpret_cast<double *>(b + L.dens_sum);
    W.phi_sum = reinterpret_cast<double *>(b + L.phi_sum);
    W.nsamp = reinterpret_cast<unsigned long long *>(b + L.nsamp);
    W.dens_sum_fix = reinterpret_cast<long long *>(b + L.dens_sum);
    W.phi_s2_sum = reinterpret_cast<__int128 *>(b + L.phi_s2_sum);
    W.phi0_sum = reinterpret_cast<double *>(b + L.phi0_sum);
    W.D0_sum = reinterpret_cast<double *>(b + L.D0_sum);
    W.counters = reinterpret_cast<unsigned long long *>(b + L.counters);
    W.eedf = reinterpret_cast<unsigned *>(b + L.eedf);
    W.iedf = reinterpret_cast<unsigned *>(b + L.iedf);
    W.fm = reinterpret_cast<unsigned *>(b + L.fm);
    W.tables = reinterpret_cast<TableDesc *>(b + L.tables);
    W.lutE = reinterpret_cast<double *>(b + L.lutE);
    W.lutS = reinterpret_cast<double *>(b + L.lutS);
    W.lutEf = reinterpret_cast<float *>(b + L.lutEf);
    W.lutSf = reinterpret_cast<float *>(b + L.lutSf);
    W.gtab = reinterpret_cast<double *>(b + L.gtab);
    W.gtabf = reinterpret_cast<float *>(b + L.gtabf);
    W.gpm = reinterpret_cast<double *>(b + L.gpm);
    W.gpmf = reinterpret_cast<float *>(b + L.gpmf);
    W.sort_counts = reinterpret_cast<int *>(b + L.sort_counts);
    W.sort_whist = reinterpret_cast<unsigned short *>(b + L.sort_whist);
    W.cell_start = reinterpret_cast<int *>(b + L.cell_start);
    W.sort_live = reinterpret_cast<int *>(b + L.sort_live);
    W.sort_tot = reinterpret_cast<int *>(b + L.sort_tot);
    W.pair_bcount = reinterpret_cast<int *>(b + L.pair_bcount);
    W.cell_disc = reinterpret_cast<int *>(b + L.cell_disc);
    W.pair_first = reinterpret_cast<int *>(b + L.pair_first);
    W.vmax2 = reinterpret_cast<unsigned long long *>(b + L.vmax2);
    W.nubin = reinterpret_cast<NuBin *>(b + L.nubin);
    W.cand = reinterpret_cast<int2 *>(b + L.cand);
    W.cand_cap = L.cand_cap;
    W.pair_kills = reinterpret_cast<int *>(b + L.pair_kills);
    W.pair_births = b + L.pair_births;
    W.total_nodes = L.total_nodes;
    W.total_cells = L.total_cells;
    W.max_chunks = L.max_chunks;
    W.D = n_discharges;
    for (int k = 0; k < 2; ++k) {
        h->Pf.cell[k] = h->Pd.cell[k] = reinterpret_cast<int *>(b + L.cell[k]);
        h->Pf.off[k] = reinterpret_cast<float *>(b + L.off[k]);
        h->Pf.vx[k] = reinterpret_cast<float *>(b + L.vx[k]);
        h->Pf.vy[k] = reinterpret_cast<float *>(b + L.vy[k]);
        h->Pf.vz[k] = reinterpret_cast<float *>(b + L.vz[k]);
        h->Pd.off[k] = reinterpret_cast<double *>(b + L.off[k]);
        h->Pd.vx[k] = reinterpret_cast<double *>(b + L.vx[k]);
        h->Pd.vy[k] = reinterpret_cast<double *>(b + L.vy[k]);
        h->Pd.vz[k] = reinterpret_cast<double *>(b + L.vz[k]);
    }
    h->sort_tab = reinterpret_cast<int *>(b + L.sort_tab);

    // tables: descriptors and LUTs
    std::vector<TableDesc> td(n_xs);
    std::vector<double> lE, lS;
    std::vector<float> lEf, lSf;
    std::vector<int> gas(3 * MAX_GAS_CH, 0), gcount(3, 0);
    int pair_tab[20];
    for (int r = 0; r < 20; ++r) pair_tab[r] = -1;
    for (int i = 0; i < n_xs; ++i) {
        const HostTable &t = h->tabs[i];
        td[i].off = (int)lE.size();
        td[i].n = t.n;
        td[i].reaction = t.reaction;
        td[i].th = t.th;
        td[i].lnE0 = std::log(t.E[0]);
        td[i].inv_dlog = (t.n - 1) / std::log(t.E[t.n - 1] / t.E[0]);
        td[i].th_f = (float)td[i].th;
        td[i].lnE0_f = (float)td[i].lnE0;
        td[i].inv_dlog_f = (float)td[i].inv_dlog;
        for (int k = 0; k < t.n; ++k) {
            lE.push_back(t.E[k]);
            lS.push_back(t.S[k]);
            lEf.push_back((float)t.E[k]);
            lSf.push_back((float)t.S[k]);
        }
        if (targ_of(t.reaction) >= 0) {
            pair_tab[t.reaction] = i;
        } else {
            const int s = proj_of(t.reaction);
            gas[s * MAX_GAS_CH + gcount[s]++] = i;
        }
    }
    h->disc.resize(n_discharges);
    h->nubin.assign((size_t)n_discharges * NUBIN_MAX, NuBin{});
    h->numax.assign(3 * n_discharges, 0.0);
    for (int d = 0; d < n_discharges; ++d) build_disc(h, d, gas, gcount, pair_tab);
    // node-major gas tables: row k of (d, s) holds n_j dx sigma_j(E_k), j < nch
    std::vector<double> gt(std::max(1LL, L.gtab_n), 0.0);
    std::vector<float> gtf(std::max(1LL, L.gtab_n), 0.0f);
    std::vector<double> gpm(std::max(1LL, L.gtab_n), 0.0);
    std::vector<float> gpmf(std::max(1LL, L.gtab_n), 0.0f);
    {
        long long off = 0;
        for (int d = 0; d < n_discharges; ++d)
            for (int s = 0; s < 3; ++s) {
                SpeciesC &S = h->disc[d].sp[s];
                const int ld = (S.nch + 3) / 4 * 4;
                const int nodes = S.nch > 0 ? h->tabs[S.ch[0].table].n : 0;
                S.gtab_ld = ld;
                S.gtab_off = (int)off;
                for (int k = 0; k < nodes; ++k)
                    for (int j = 0; j < S.nch; ++j) {
                        const double v = S.ch[j].coef * h->tabs[S.ch[j].table].S[k];
                        gt[off + (long long)k * ld + j] = v;
                        gtf[off + (long long)k * ld + j] = (float)v;
                    }
                // bound for the sequential scheme's skip: row k holds the largest
                // max(v_i, v_{i+1}) u_n(E_{i+1}) over the intervals i <= k (v linear
                // between nodes, u_n = sqrt(E / Ek) increasing), row nodes-1 repeats
                // row nodes-2
                for (int j = 0; j < S.nch; ++j) {
                    double run = 0.0;
                    const HostTable &t = h->tabs[S.ch[j].table];
                    for (int k = 0; k < nodes; ++k) {
                        if (k + 1 < nodes) {
                            const double u1 = std::sqrt(t.E[k + 1] / S.Ek);
                            const double a = gt[off + (long long)k * ld + j], c2 = gt[off + (long long)(k + 1) * ld + j];
                            run = std::max(run, std::max(a, c2) * u1);
                        }
                        gpm[off + (long long)k * ld + j] = run;
                        gpmf[off + (long long)k * ld + j] = (float)run;
                    }
                }
                off += (long long)nodes * ld + 4;
            }
    }

    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    h->L.maxN = L.maxN;
    h->L.eedf_max = L.eedf_max;
    h->L.fm_max = L.fm_max;
    h->L.sort_blocks = L.sort_blocks;
    h->L.sort_warp_base = reinterpret_cast<const int *>(b + L.warp_base);
    std::vector<int> wbase(3 * n_discharges + 1, 0);
    for (int d = 0; d < n_discharges; ++d)
        for (int s = 0; s < 3; ++s) {
            // column-scan warps of (d, s): groups of 32 buckets x segments of rows
            const int g = L.sort_gmax[3 * d + s];
            wbase[3 * d + s + 1] = wbase[3 * d + s] +
                                   ((cfgs[d].n_cells + 1 + 31) / 32) * ((g + COLSCAN_SEG - 1) / COLSCAN_SEG);
        }
    h->L.sort_col_warps = wbase[3 * n_discharges];
    CK(configure_kernels(h->fp64, h->L));
    CK(push_configure(h->fp64, h->L, nsm));

    // host-built small tables
    std::vector<int> stab;
    std::vector<int> cdisc(L.total_cells);
    for (int d = 0; d < n_discharges; ++d) {
        for (int s = 0; s < 3; ++s)
            for (int g = 0; g < L.sort_gmax[3 * d + s]; ++g) {
                stab.push_back(3 * d + s);
                stab.push_back(g);
            }
        for (int c = 0; c < h->cfg[d].n_cells; ++c) cdisc[L.ccell[d] + c] = d;
    }
    std::vector<long long> ninit(3 * n_discharges);
    std::vector<double> vt(3 * n_discharges);
    std::vector<Counts> cnt(3 * n_discharges);
    int max_n = 1;
    for (int d = 0; d < n_discharges; ++d)
        for (int s = 0; s < 3; ++s) {
            ninit[3 * d + s] = h->cfg[d].n_init[s];
            vt[3 * d + s] = std::sqrt(h->cfg[d].T0_eV[s] * QE / MASS[s]);
            cnt[3 * d + s] = Counts{(int)h->cfg[d].n_init[s], 0, 0, 0};
            max_n = std::max(max_n, (int)h->cfg[d].n_init[s]);
        }
    Ctl ctl{};
    ctl.D = n_discharges;
    cudaStream_t st = h->stream;
    CK(cudaMemsetAsync(h->ws, 0, L.total, st));
    CK(cudaMemcpyAsync(W.ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(W.disc, h->disc.data(), sizeof(Disc) * n_discharges, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(W.nubin, h->nubin.data(), sizeof(NuBin) * h->nubin.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(W.cnt, cnt.data(), sizeof(Counts) * cnt.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(W.gtab, gt.data(), 8 * gt.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(W.gtabf, gtf.data(), 4 * gtf.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(W.gpm, gpm.data(), 8 * gpm.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(W.gpmf, gpmf.data(), 4 * gpmf.size(), cudaMemcpyHostToDevice, st));
    if (n_xs > 0) {
        CK(cudaMemcpyAsync(W.tables, td.data(), sizeof(TableDesc) * n_xs, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(W.lutE, lE.data(), 8 * lE.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(W.lutS, lS.data(), 8 * lS.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(W.lutEf, lEf.data(), 4 * lEf.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(W.lutSf, lSf.data(), 4 * lSf.size(), cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(h->sort_tab, stab.data(), 4 * stab.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(W.cell_disc, cdisc.data(), 4 * cdisc.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b + L.warp_base, wbase.data(), 4 * wbase.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(W.pair_first, 0x7F, 4ull * L.total_cells, st));
    for (int s = 0; s < 3; ++s) {
        std::vector<int> pt;
        for (int d = 0; d < n_discharges; ++d)
            for (long long t = 0; t < (h->cfg[d].capacity[s] + 255) / 256; ++t) {
                pt.push_back(d);
                pt.push_back((int)t);
            }
        h->L.pair_blocks_sp[s] = (int)(pt.size() / 2);
        h->L.pair_tab_sp[s] = reinterpret_cast<const int *>(b + L.pair_tab[s]);
        if (!pt.empty())
            CK(cudaMemcpyAsync(b + L.pair_tab[s], pt.data(), 4 * pt.size(), cudaMemcpyHostToDevice, st));
    }
    long long *d_ninit = reinterpret_cast<long long *>(b + L.ninit);
    double *d_vt = reinterpret_cast<double *>(b + L.vt);
    CK(cudaMemcpyAsync(d_ninit, ninit.data(), 8 * ninit.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_vt, vt.data(), 8 * vt.size(), cudaMemcpyHostToDevice, st));
    CK(launch_load(h->fp64, W, h->pools(), d_ninit, d_vt, max_n, st));
    CK(launch_deposit_all(h->fp64, W, h->pools(), -1, max_n, st));
    CK(cudaStreamSynchronize(st));
    h->launches = 0;
    *out = h;
    return PIC_OK;
}

static long long lcm_ll(long long a, long long b) { return a / std::gcd(a, b) * b; }

// Kernels of one step; returns the number launched.
// events around one kernel launch in timing mode (kind 0 push, 1 Coulomb)
static cudaError_t time_open(pic_handle *h, bool on, cudaStream_t st)
{
    if (!on) return cudaSuccess;
    if (h->ev_used + 2 > (int)h->ev.size()) return cudaErrorNotReady;
    return cudaEventRecord(h->ev[h->ev_used], st);
}

static cudaError_t time_close(pic_handle *h, bool on, cudaStream_t st, int kind)
{
    if (!on) return cudaSuccess;
    cudaError_t e = cudaEventRecord(h->ev[h->ev_used + 1], st);
    if (e) return e;
    h->ev_kind[h->ev_used / 2] = kind;
    h->ev_used += 2;
    return cudaSuccess;
}

static cudaError_t enqueue_step(pic_handle *h, long long n, int &nk, bool timed)
{
    const pic_config &q = h->cfg[0];
    const int par = (int)(n & 1);
    const bool diag = q.diag_every > 0 && (n % q.diag_every) == 0;
    cudaStream_t st = h->stream;
    cudaError_t e = launch_field(h->fp64, diag, 0, h->W, par, h->L, st);
    if (e) return e;
    ++nk;
    if ((e = time_open(h, timed, st))) return e;
    e = launch_push(h->fp64, diag, h->W, h->pools(), par, h->L, st);
    if (e) return e;
    ++nk;
    if ((e = time_close(h, timed, st, diag ? PIC_KERNEL_PUSH_DIAG : PIC_KERNEL_PUSH))) return e;
    e = launch_collide(h->fp64, h->W, h->pools(), par, h->L.collide_blocks, st);
    if (e) return e;
    ++nk;
    e = launch_births(h->fp64, h->W, h->pools(), par, h->W.max_chunks / TILE_ALIGN + 1, st);
    if (e) return e;
    ++nk;
    const long long next = n + 1;
    const bool pair = q.n1 > 0 && next % q.n1 == 0;
    const bool coul = q.n2 > 0 && next % q.n2 == 0;
    const bool sort = pair || coul || (q.sort_interval > 0 && next % q.sort_interval == 0);
    if (sort) {
        e = launch_sort(h->fp64, h->W, h->pools(), h->sort_tab, h->L, st);
        if (e) return e;
        nk += kernels_per_sort();
    }
    if (coul) {
        if ((e = time_open(h, timed, st))) return e;
        e = launch_coulomb(h->fp64, h->W, h->pools(), par, st);
        if (e) return e;
        ++nk;
        if (q.coulomb_inter) {
            for (int pr = 0; pr < 3; ++pr)
                if ((e = launch_coulomb_inter(h->fp64, h->W, h->pools(), par, pr, st))) return e;
            nk += 3;
        }
        if ((e = time_close(h, timed, st, 1))) return e;
    }
    if (pair && q.gas_scheme == 1) {
        // the sequential scheme (R22): gas channels below (13), (13), (14),
        // gas channels above (14), their births, a new sort, (19)
        if ((e = launch_retile(h->W, par, st))) return e;
        if ((e = time_open(h, timed, st))) return e;
        if ((e = launch_dsmc(h->fp64, h->W, h->pools(), par, 0, st))) return e;
        if ((e = time_close(h, timed, st, 2))) return e;
        if ((e = launch_pair_reaction(h->fp64, h->W, h->pools(), par, 0, st))) return e;
        if ((e = launch_pair_reaction(h->fp64, h->W, h->pools(), par, 1, st))) return e;
        if ((e = time_open(h, timed, st))) return e;
        if ((e = launch_dsmc(h->fp64, h->W, h->pools(), par, 1, st))) return e;
        if ((e = time_close(h, timed, st, 2))) return e;
        if ((e = launch_births(h->fp64, h->W, h->pools(), par, h->W.max_chunks / TILE_ALIGN + 1, st, 1))) return e;
        if ((e = launch_sort(h->fp64, h->W, h->pools(), h->sort_tab, h->L, st))) return e;
        // the kill counts of (13), (14) refer to the cells before the sort
        if ((e = cudaMemsetAsync(h->W.pair_kills, 0, sizeof(int) * NSP * (size_t)h->W.total_cells, st))) return e;
        if ((e = launch_pair_reaction(h->fp64, h->W, h->pools(), par, 2, st))) return e;
        if ((e = launch_pair_append(h->fp64, h->W, h->pools(), h->L, st))) return e;
        nk += 1 + 2 + 2 * 3 + 1 + kernels_per_sort() + 1;
    } else if (pair) {
        e = launch_pair(h->fp64, h->W, h->pools(), par, h->L, st);
        if (e) return e;
        nk += kernels_per_pair();
    }
    return cudaSuccess;
}

static pic_status harvest_events(pic_handle *h)
{
    if (h->ev_used == 0) return PIC_OK;
    CK(cudaEventSynchronize(h->ev[h->ev_used - 1]));
    for (int i = 0; i < h->ev_used; i += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]));
        const int k = h->ev_kind[i / 2];
        h->kms[k] += ms;
        h->kl[k] += 1;
    }
    h->ev_used = 0;
    return PIC_OK;
}

static pic_status check_status(pic_handle *h)
{
    unsigned status = 0;
    CK(cudaMemcpyAsync(&status, &h->W.ctl->status, sizeof status, cudaMemcpyDeviceToHost, h->stream));
    std::vector<unsigned long long> c((size_t)h->D * C_NCOUNT);
    CK(cudaMemcpyAsync(c.data(), h->W.counters, 8 * c.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (status & ST_TIMEOUT) return fail(h, PIC_ETIMEOUT, "a bounded device wait (birth look-back) gave up");
    if (status & (ST_CAPACITY | ST_BIRTHBUF))
        return fail(h, PIC_ECAPACITY, (status & ST_CAPACITY) ? "particle capacity exceeded; births were dropped"
                                                             : "a per-chunk or per-cell birth buffer overflowed");
    if (status & ST_BADSTATE) return fail(h, PIC_EINVAL, "inconsistent device state");
    if (status & ST_NONFINITE)
        return fail(h, PIC_ENUMERIC, "a particle position or velocity became non-finite (the particle was removed)");
    for (int d = 0; d < h->D; ++d) {
        const unsigned long long *cd = &c[(size_t)d * C_NCOUNT];
        if (cd[C_VIOL_GAS] > 10 && (double)cd[C_VIOL_GAS] > h->numeric_budget * (double)cd[C_CANDS])
            return fail(h, PIC_ENUMERIC, "collision frequency above nu_max too often (raise ecap_eV)");
        if (cd[C_VIOL_PAIR] > 10 && (double)cd[C_VIOL_PAIR] > h->numeric_budget * (double)cd[C_PEVAL])
            return fail(h, PIC_ENUMERIC, "Eq. 1 probability above 1 too often (shorten n1 dt)");
    }
    return PIC_OK;
}

// Capture `nsteps` time steps from the current step as one CUDA graph (on a
// private stream, thread-local capture); false if capture or instantiation
// failed.
static bool capture_steps(pic_handle *h, long long nsteps, cudaGraphExec_t *out, long long *kernels)
{
    cudaGraph_t g = nullptr;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int nk = 0;
    cudaStream_t keep = h->stream;
    h->stream = cs;
    for (long long k = 0; ok && k < nsteps; ++k) ok = enqueue_step(h, h->step + k, nk, false) == cudaSuccess;
    h->stream = keep;
    cudaError_t ee = cudaStreamEndCapture(cs, &g);
    ok = ok && ee == cudaSuccess && g;
    if (ok) ok = cudaGraphInstantiate(out, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (!ok) *out = nullptr;
    *kernels = nk;
    return ok;
}

// the longest stretch captured as one graph
constexpr long long MAX_GRAPH_STEPS = 8192;

extern "C" pic_status pic_step(pic_handle *h, long long n_steps)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    if (n_steps < 0) return fail(h, PIC_EINVAL, "n_steps < 0");
    const pic_config &q = h->cfg[0];
    if (h->period == 0) {
        long long P = 2;
        if (q.n1 > 0) P = lcm_ll(P, q.n1);
        if (q.n2 > 0) P = lcm_ll(P, q.n2);
        if (q.sort_interval > 0) P = lcm_ll(P, q.sort_interval);
        if (q.diag_every > 0) P = lcm_ll(P, q.diag_every);
        h->period = P;
        // one RF cycle as the graph unit when it is a whole number of time
        // steps and of schedule periods (the drive phase is read on the
        // device from the step counter, so any period-aligned start replays
        // the same work)
        const double spc = 1.0 / (q.f_rf_Hz * q.dt_s);
        const long long c = std::llround(spc);
        h->cycle_steps = 0;
        if (c >= P && std::fabs(spc - (double)c) <= 1e-6 * spc && c % P == 0 && c <= MAX_GRAPH_STEPS)
            h->cycle_steps = c;
    }
    long long left = n_steps;
    while (left > 0) {
        const bool aligned = (h->step % h->period) == 0;
        const bool graphs = !h->timing && !h->graph_failed && aligned;
        if (graphs && h->cycle_steps > 0 && left >= h->cycle_steps) {
            if (!h->gexec_cycle) {
                if (!capture_steps(h, h->cycle_steps, &h->gexec_cycle, &h->cycle_graph_launches)) {
                    h->graph_failed = true;
                    continue;
                }
            }
            CK(cudaGraphLaunch(h->gexec_cycle, h->stream));
            ++h->graph_calls;
            h->launches += h->cycle_graph_launches;
            h->step += h->cycle_steps;
            left -= h->cycle_steps;
            continue;
        }
        if (graphs && left >= h->period && h->period <= MAX_GRAPH_STEPS) {
            if (!h->gexec) {
                if (!capture_steps(h, h->period, &h->gexec, &h->graph_launches)) {
                    h->graph_failed = true;
                    continue;
                }
            }
            CK(cudaGraphLaunch(h->gexec, h->stream));
            ++h->graph_calls;
            h->launches += h->graph_launches;
            h->step += h->period;
            left -= h->period;
            continue;
        }
        int nk = 0;
        if (h->timing && h->ev_used + 8 > (int)h->ev.size()) {
            pic_status s = harvest_events(h);
            if (s != PIC_OK) return s;
        }
        cudaError_t e = enqueue_step(h, h->step, nk, h->timing);
        if (e) return cuda_fail(h, e, "kernel launch");
        h->launches += nk;
        h->step += 1;
        left -= 1;
    }
    if (h->timing) {
        pic_status s = harvest_events(h);
        if (s != PIC_OK) return s;
    }
    return check_status(h);
}

extern "C" pic_status pic_set_numeric_budget(pic_handle *h, double max_fraction)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    if (!(max_fraction >= 0.0) || !(max_fraction <= 1.0))
        return fail(h, PIC_EINVAL, "max_fraction must lie in [0, 1]");
    h->numeric_budget = max_fraction;
    return PIC_OK;
}

extern "C" pic_status pic_set_step(pic_handle *h, long long step)
{
    if (!h || step < 0) return fail(h, PIC_EINVAL, "bad handle or step");
    unsigned long long v = (unsigned long long)step;
    CK(cudaMemcpyAsync(&h->W.ctl->step[step & 1], &v, 8, cudaMemcpyHostToDevice, h->stream));
    // look-back words are tagged with the step; a step number can now repeat
    CK(cudaMemsetAsync(h->W.births_lb, 0, 8ull * 3 * (h->W.max_chunks / TILE_ALIGN + 1), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->step = step;
    return PIC_OK;
}

extern "C" pic_status pic_diagnostics(pic_handle *h, int d, double *dens_sum, double *phi_sum, long long *eedf,
                                      long long *iedf, long long *fm, long long *counters, long long *n_samples,
                                      int reset)
{
    if (!h || d < 0 || d >= h->D) return fail(h, PIC_EINVAL, "bad handle or discharge");
    const pic_config &q = h->cfg[d];
    const Disc &D = h->disc[d];
    const int N = q.n_cells, tn = h->W.total_nodes;
    cudaStream_t st = h->stream;
    // FP32 path: exact integer sums, scaled here; FP64 path: FP64 sums
    std::vector<long long> dfix(h->fp64 ? 0 : 3 * (size_t)(N + 1));
    std::vector<__int128> s2(h->fp64 ? 0 : (size_t)(N + 1));
    double p0s = 0.0, d0s = 0.0;
    if (dens_sum) {
        for (int s = 0; s < 3; ++s) {
            if (h->fp64)
                CK(cudaMemcpyAsync(dens_sum + (size_t)s * (N + 1), h->W.dens_sum + (size_t)s * tn + D.gbase,
                                   8 * (N + 1), cudaMemcpyDeviceToHost, st));
            else
                CK(cudaMemcpyAsync(dfix.data() + (size_t)s * (N + 1), h->W.dens_sum_fix + (size_t)s * tn + D.gbase,
                                   8 * (N + 1), cudaMemcpyDeviceToHost, st));
        }
    }
    if (phi_sum) {
        if (h->fp64) {
            CK(cudaMemcpyAsync(phi_sum, h->W.phi_sum + D.gbase, 8 * (N + 1), cudaMemcpyDeviceToHost, st));
        } else {
            CK(cudaMemcpyAsync(s2.data(), h->W.phi_s2_sum + D.gbase, 16 * (N + 1), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(&p0s, h->W.phi0_sum + d, 8, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(&d0s, h->W.D0_sum + d, 8, cudaMemcpyDeviceToHost, st));
        }
    }
    std::vector<unsigned> e(std::max(1, q.eedf_bins)), i2(std::max(1, 2 * q.iedf_bins)),
        f(std::max(1, D.fm_xbins * q.fm_bins));
    if (q.eedf_bins)
        CK(cudaMemcpyAsync(e.data(), h->W.eedf + D.eedf_base, 4 * q.eedf_bins, cudaMemcpyDeviceToHost, st));
    if (q.iedf_bins)
        CK(cudaMemcpyAsync(i2.data(), h->W.iedf + D.iedf_base, 8 * q.iedf_bins, cudaMemcpyDeviceToHost, st));
    if (q.fm_bins)
        CK(cudaMemcpyAsync(f.data(), h->W.fm + D.fm_base, 4 * (size_t)D.fm_xbins * q.fm_bins,
                           cudaMemcpyDeviceToHost, st));
    std::vector<unsigned long long> c(C_NCOUNT);
    CK(cudaMemcpyAsync(c.data(), h->W.counters + (size_t)d * C_NCOUNT, 8 * C_NCOUNT, cudaMemcpyDeviceToHost, st));
    unsigned long long ns = 0;
    CK(cudaMemcpyAsync(&ns, h->W.nsamp + d, 8, cudaMemcpyDeviceToHost, st));
    Counts cn[3];
    CK(cudaMemcpyAsync(cn, h->W.cnt + 3 * d, sizeof cn, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!h->fp64 && dens_sum)
        for (int s = 0; s < 3; ++s)
            for (int i = 0; i <= N; ++i)
                dens_sum[(size_t)s * (N + 1) + i] =
                    (double)dfix[(size_t)s * (N + 1) + i] * ((i == 0 || i == N) ? D.dens_fix_wall : D.dens_fix);
    if (!h->fp64 && phi_sum) {
        const double Kdx = 1.602176634e-19 * q.weight_m2 / (double)(1 << FIX_BITS) / 8.8541878128e-12 * D.dx;
        phi_sum[0] = p0s;
        phi_sum[N] = 0.0;
        for (int i = 1; i < N; ++i) phi_sum[i] = p0s + (double)i * d0s - Kdx * (double)s2[i];
    }
    if (eedf) for (int k = 0; k < q.eedf_bins; ++k) eedf[k] = e[k];
    if (iedf) for (int k = 0; k < 2 * q.iedf_bins; ++k) iedf[k] = i2[k];
    if (fm) for (int k = 0; k < D.fm_xbins * q.fm_bins; ++k) fm[k] = f[k];
    if (counters) {
        for (int k = 0; k < 28; ++k) counters[k] = (long long)c[k];
        for (int s = 0; s < 3; ++s) counters[28 + s] = cn[s].n;
        counters[31] = h->step;
        counters[32] = (long long)c[C_LIVE];
        counters[33] = (long long)c[C_CANDS];
        counters[34] = (long long)c[C_SLOTS];
        counters[35] = (long long)c[C_COUL];
        counters[36] = (long long)c[C_DSMC];
        counters[37] = (long long)c[C_PEVAL];
        counters[38] = h->cycle_steps;
        counters[39] = h->graph_calls;
    }
    if (n_samples) *n_samples = (long long)ns;
    if (reset) {
        for (int s = 0; s < 3; ++s)
            CK(cudaMemsetAsync(h->W.dens_sum + (size_t)s * tn + D.gbase, 0, 8 * (N + 1), st));
        CK(cudaMemsetAsync(h->W.phi_sum + D.gbase, 0, 8 * (N + 1), st));
        CK(cudaMemsetAsync(h->W.phi_s2_sum + D.gbase, 0, 16 * (N + 1), st));
        CK(cudaMemsetAsync(h->W.phi0_sum + d, 0, 8, st));
        CK(cudaMemsetAsync(h->W.D0_sum + d, 0, 8, st));
        if (q.eedf_bins) CK(cudaMemsetAsync(h->W.eedf + D.eedf_base, 0, 4 * q.eedf_bins, st));
        if (q.iedf_bins) CK(cudaMemsetAsync(h->W.iedf + D.iedf_base, 0, 8 * q.iedf_bins, st));
        if (q.fm_bins) CK(cudaMemsetAsync(h->W.fm + D.fm_base, 0, 4 * (size_t)D.fm_xbins * q.fm_bins, st));
        CK(cudaMemsetAsync(h->W.nsamp + d, 0, 8, st));
        CK(cudaStreamSynchronize(st));
    }
    return PIC_OK;
}

extern "C" pic_status pic_get_state(pic_handle *h, int d, int s, double *x, double *vx, double *vy, double *vz,
                                    int *alive, long long capacity_n, long long *n)
{
    if (!h || d < 0 || d >= h->D || s < 0 || s > 2) return fail(h, PIC_EINVAL, "bad handle, discharge or species");
    Counts cn;
    int cur = 0;
    CK(cudaMemcpyAsync(&cn, h->W.cnt + 3 * d + s, sizeof cn, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&cur, &h->W.ctl->cur, sizeof cur, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (n) *n = cn.n;
    if (!x && !vx && !vy && !vz && !alive) return PIC_OK;
    if (capacity_n < cn.n) return fail(h, PIC_EINVAL, "host arrays shorter than the slot count");
    const Disc &D = h->disc[d];
    const size_t g = D.pbase[s], m = cn.n;
    const size_t R = h->fp64 ? 8 : 4;
    const char *base = h->ws;
    const Layout &L = h->lay;
    std::vector<int> cell(m);
    std::vector<char> o(m * R), a(m * R), bb(m * R), cc(m * R);
    if (m) {
        CK(cudaMemcpyAsync(cell.data(), base + L.cell[cur] + 4 * g, 4 * m, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(o.data(), base + L.off[cur] + R * g, R * m, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(a.data(), base + L.vx[cur] + R * g, R * m, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(bb.data(), base + L.vy[cur] + R * g, R * m, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(cc.data(), base + L.vz[cur] + R * g, R * m, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    const double dx = D.dx, vs = D.dx / D.dt;
    auto rd = [&](const std::vector<char> &v, size_t i) {
        return h->fp64 ? reinterpret_cast<const double *>(v.data())[i]
                       : (double)reinterpret_cast<const float *>(v.data())[i];
    };
    for (size_t i = 0; i < m; ++i) {
        const bool al = cell[i] >= 0;
        if (x) x[i] = al ? ((double)cell[i] + rd(o, i)) * dx : 0.0;
        if (vx) vx[i] = rd(a, i) * vs;
        if (vy) vy[i] = rd(bb, i) * vs;
        if (vz) vz[i] = rd(cc, i) * vs;
        if (alive) alive[i] = al ? 1 : 0;
    }
    return PIC_OK;
}

extern "C" pic_status pic_set_state(pic_handle *h, int d, int s, long long n, const double *x, const double *vx,
                                    const double *vy, const double *vz, const int *alive)
{
    if (!h || d < 0 || d >= h->D || s < 0 || s > 2) return fail(h, PIC_EINVAL, "bad handle, discharge or species");
    if (n < 0 || n > h->cfg[d].capacity[s]) return fail(h, PIC_ECAPACITY, "n exceeds the species capacity");
    if (n > 0 && (!x || !vx || !vy || !vz)) return fail(h, PIC_EINVAL, "NULL state array");
    const Disc &D = h->disc[d];
    const int N = D.N;
    const size_t R = h->fp64 ? 8 : 4;
    std::vector<int> cell(n);
    std::vector<char> o(n * R), a(n * R), bb(n * R), cc(n * R);
    const double tdx = D.dt / D.dx;
    for (long long i = 0; i < n; ++i) {
        const bool al = alive ? alive[i] != 0 : true;
        const double xx = x[i] / D.dx;
        int c = al ? (int)std::floor(xx) : -1;
        if (al && (!(x[i] >= 0.0) || !(x[i] < D.L))) return fail(h, PIC_EINVAL, "live particle outside [0, L)");
        if (c > N - 1) c = N - 1;
        double off = al ? xx - c : 0.0;
        if (h->fp64) {
            reinterpret_cast<double *>(o.data())[i] = off;
            reinterpret_cast<double *>(a.data())[i] = vx[i] * tdx;
            reinterpret_cast<double *>(bb.data())[i] = vy[i] * tdx;
            reinterpret_cast<double *>(cc.data())[i] = vz[i] * tdx;
        } else {
            float of = (float)off;
            if (al && of >= 1.0f) {
                if (c + 1 < N) {
                    ++c;
                    of = 0.0f;
                } else {
                    of = std::nextafter(1.0f, 0.0f);
                }
            }
            reinterpret_cast<float *>(o.data())[i] = of;
            reinterpret_cast<float *>(a.data())[i] = (float)(vx[i] * tdx);
            reinterpret_cast<float *>(bb.data())[i] = (float)(vy[i] * tdx);
            reinterpret_cast<float *>(cc.data())[i] = (float)(vz[i] * tdx);
        }
        cell[i] = c;
    }
    int cur = 0;
    CK(cudaMemcpyAsync(&cur, &h->W.ctl->cur, sizeof cur, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const size_t g = D.pbase[s];
    char *base = h->ws;
    const Layout &L = h->lay;
    if (n) {
        CK(cudaMemcpyAsync(base + L.cell[cur] + 4 * g, cell.data(), 4 * n, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(base + L.off[cur] + R * g, o.data(), R * n, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(base + L.vx[cur] + R * g, a.data(), R * n, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(base + L.vy[cur] + R * g, bb.data(), R * n, cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(base + L.vz[cur] + R * g, cc.data(), R * n, cudaMemcpyHostToDevice, h->stream));
    }
    Counts cn{(int)n, 0, 0, 0};
    CK(cudaMemcpyAsync(h->W.cnt + 3 * d + s, &cn, sizeof cn, cudaMemcpyHostToDevice, h->stream));
    const int tn = h->W.total_nodes;
    for (int sp = 0; sp < 3; ++sp)
        CK(cudaMemsetAsync(reinterpret_cast<char *>(h->W.acc_dbl) + 8 * ((size_t)sp * tn + D.gbase), 0,
                           8 * (N + 1), h->stream));
    int max_n = 1;
    for (int sp = 0; sp < 3; ++sp) max_n = std::max(max_n, (int)h->cfg[d].capacity[sp]);
    CK(launch_deposit_all(h->fp64, h->W, h->pools(), d, max_n, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

extern "C" pic_status pic_fields(pic_handle *h, int d, double *rho, double *phi, double *E)
{
    if (!h || d < 0 || d >= h->D) return fail(h, PIC_EINVAL, "bad handle or discharge");
    CK(launch_field(h->fp64, false, 1, h->W, (int)(h->step & 1), h->L, h->stream));
    const Disc &D = h->disc[d];
    const int N = D.N;
    if (rho) CK(cudaMemcpyAsync(rho, h->W.rho + D.gbase, 8 * (N + 1), cudaMemcpyDeviceToHost, h->stream));
    if (phi) CK(cudaMemcpyAsync(phi, h->W.phi + D.gbase, 8 * (N + 1), cudaMemcpyDeviceToHost, h->stream));
    if (E) CK(cudaMemcpyAsync(E, h->W.Efield + D.gbase, 8 * (N + 1), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return PIC_OK;
}

extern "C" double pic_numax(const pic_handle *h, int d, int s)
{
    if (!h || d < 0 || d >= h->D || s < 0 || s > 2) return -1.0;
    return h->numax[3 * d + s];
}

extern "C" pic_status pic_set_timing(pic_handle *h, int on)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    if (on && h->ev.empty()) {
        h->ev.resize(4096);
        h->ev_kind.assign(2048, 0);
        for (auto &e : h->ev) CK(cudaEventCreate(&e));
    }
    h->timing = on != 0;
    return PIC_OK;
}

extern "C" pic_status pic_timing(pic_handle *h, double *push_ms, long long *push_launches, long long *launches,
                                 double *push_bytes, int reset)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    std::vector<unsigned long long> c((size_t)h->D * C_NCOUNT);
    CK(cudaMemcpyAsync(c.data(), h->W.counters, 8 * c.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    unsigned long long slots = 0, cands = 0, bslots = 0, bcands = 0;
    for (int d = 0; d < h->D; ++d) {
        slots += c[(size_t)d * C_NCOUNT + C_SLOTS];
        cands += c[(size_t)d * C_NCOUNT + C_CANDS];
        bslots += c[(size_t)d * C_NCOUNT + C_BSLOTS];
        bcands += c[(size_t)d * C_NCOUNT + C_BCANDS];
    }
    // algorithmic bytes of the push: cell, offset and vx read and written for
    // every slot; vy, vz read for every slot of a species whose bound depends
    // on the lab energy; one 8-byte list entry per collision candidate (the
    // collisions themselves run in the next kernel)
    const double R = h->fp64 ? 8.0 : 4.0;
    const double bytes = (double)(slots - h->slots0) * 2.0 * (4.0 + 2.0 * R) +
                         (double)(bslots - h->bslots0) * 2.0 * R + (double)(cands - h->cands0) * 8.0;
    if (push_ms) *push_ms = h->kms[PIC_KERNEL_PUSH] + h->kms[PIC_KERNEL_PUSH_DIAG];
    if (push_launches) *push_launches = h->kl[PIC_KERNEL_PUSH] + h->kl[PIC_KERNEL_PUSH_DIAG];
    if (launches) *launches = h->launches;
    if (push_bytes) *push_bytes = bytes;
    if (reset) {
        h->kms[PIC_KERNEL_PUSH] = h->kms[PIC_KERNEL_PUSH_DIAG] = 0.0;
        h->kl[PIC_KERNEL_PUSH] = h->kl[PIC_KERNEL_PUSH_DIAG] = 0;
        h->launches = 0;
        h->slots0 = slots;
        h->cands0 = cands;
        h->bslots0 = bslots;
        h->bcands0 = bcands;
    }
    return PIC_OK;
}

extern "C" pic_status pic_get_launch(pic_handle *h, int kernel, int *blocks_per_sm, int *max_blocks_per_sm)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    if (kernel != PIC_KERNEL_PUSH) return fail(h, PIC_EINVAL, "only the push has a launch shape");
    if (blocks_per_sm) *blocks_per_sm = h->L.push_per_sm;
    if (max_blocks_per_sm) *max_blocks_per_sm = h->L.push_max_per_sm;
    return PIC_OK;
}

extern "C" pic_status pic_set_launch(pic_handle *h, int kernel, int blocks_per_sm)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    if (kernel != PIC_KERNEL_PUSH) return fail(h, PIC_EINVAL, "only the push has a launch shape");
    if (blocks_per_sm < 1 || blocks_per_sm > h->L.push_max_per_sm)
        return fail(h, PIC_EINVAL, "blocks per SM out of 1 .. " + std::to_string(h->L.push_max_per_sm));
    if (blocks_per_sm == h->L.push_per_sm) return PIC_OK;
    // the captured period holds the old grid: wait for it, then drop it
    CK(cudaStreamSynchronize(h->stream));
    if (h->gexec) {
        CK(cudaGraphExecDestroy(h->gexec));
        h->gexec = nullptr;
    }
    if (h->gexec_cycle) {
        CK(cudaGraphExecDestroy(h->gexec_cycle));
        h->gexec_cycle = nullptr;
    }
    h->L.push_per_sm = blocks_per_sm;
    h->L.push_blocks = h->L.num_sms * blocks_per_sm;
    return PIC_OK;
}

extern "C" int pic_launch_shapes(pic_handle *h, int kernel, int *threads, int *slots_per_thread,
                                 int *max_blocks_per_sm, int capacity)
{
    if (!h) {
        fail(nullptr, PIC_EINVAL, "NULL handle");
        return -1;
    }
    if (kernel != PIC_KERNEL_PUSH) {
        fail(h, PIC_EINVAL, "only the push has a launch shape");
        return -1;
    }
    const int n = h->L.push_nshapes;
    for (int k = 0; k < n && k < capacity; ++k) {
        if (threads) threads[k] = h->L.shape_threads[k];
        if (slots_per_thread) slots_per_thread[k] = h->L.shape_spt[k];
        if (max_blocks_per_sm) max_blocks_per_sm[k] = h->L.shape_max_per_sm[k];
    }
    return n;
}

extern "C" pic_status pic_get_launch_shape(pic_handle *h, int kernel, int *shape, int *blocks_per_sm)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    if (kernel != PIC_KERNEL_PUSH) return fail(h, PIC_EINVAL, "only the push has a launch shape");
    if (shape) *shape = h->L.push_shape;
    if (blocks_per_sm) *blocks_per_sm = h->L.push_per_sm;
    return PIC_OK;
}

extern "C" pic_status pic_set_launch_shape(pic_handle *h, int kernel, int shape, int blocks_per_sm)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    if (kernel != PIC_KERNEL_PUSH) return fail(h, PIC_EINVAL, "only the push has a launch shape");
    if (shape < 0 || shape >= h->L.push_nshapes)
        return fail(h, PIC_EINVAL, "shape out of 0 .. " + std::to_string(h->L.push_nshapes - 1));
    const int mx = h->L.shape_max_per_sm[shape];
    if (blocks_per_sm < 1 || blocks_per_sm > mx)
        return fail(h, PIC_EINVAL, "blocks per SM out of 1 .. " + std::to_string(mx));
    if (shape == h->L.push_shape && blocks_per_sm == h->L.push_per_sm) return PIC_OK;
    // the captured graph holds the old grid: wait for it, then drop it
    CK(cudaStreamSynchronize(h->stream));
    if (h->gexec) {
        CK(cudaGraphExecDestroy(h->gexec));
        h->gexec = nullptr;
    }
    if (h->gexec_cycle) {
        CK(cudaGraphExecDestroy(h->gexec_cycle));
        h->gexec_cycle = nullptr;
    }
    h->L.push_shape = shape;
    h->L.push_max_per_sm = mx;
    h->L.push_smem = h->L.shape_smem[shape];
    h->L.push_smem_diag = h->L.shape_smem_diag[shape];
    h->L.push_per_sm = blocks_per_sm;
    h->L.push_blocks = h->L.num_sms * blocks_per_sm;
    return PIC_OK;
}

extern "C" pic_status pic_kernel_timing(pic_handle *h, int kernel, double *ms, long long *launches,
                                        double *bytes, int reset)
{
    if (!h) return fail(nullptr, PIC_EINVAL, "NULL handle");
    if (kernel == PIC_KERNEL_PUSH || kernel == PIC_KERNEL_PUSH_DIAG) {
        // the push launches of one kind; the algorithmic bytes are shared out
        // by launches (every launch of a step moves the same particle data)
        const double kms = h->kms[kernel];
        const long long kl = h->kl[kernel];
        long long all = 0, pl = 0;
        double pms = 0.0, pbytes = 0.0;
        const pic_status st = pic_timing(h, &pms, &pl, &all, &pbytes, 0);
        if (st != PIC_OK) return st;
        if (ms) *ms = kms;
        if (launches) *launches = kl;
        if (bytes) *bytes = pl > 0 ? pbytes * (double)kl / (double)pl : 0.0;
        if (reset) {
            long long a2 = 0, l2 = 0;
            double m2 = 0.0, b2 = 0.0;
            return pic_timing(h, &m2, &l2, &a2, &b2, 1);
        }
        return PIC_OK;
    }
    if (kernel != PIC_KERNEL_COULOMB && kernel != PIC_KERNEL_SEQUENTIAL_GAS)
        return fail(h, PIC_EINVAL, "unknown kernel kind");
    std::vector<unsigned long long> c((size_t)h->D * C_NCOUNT);
    CK(cudaMemcpyAsync(c.data(), h->W.counters, 8 * c.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const int slot = kernel == PIC_KERNEL_COULOMB ? C_COUL : C_DSMC;
    unsigned long long units = 0;
    for (int d = 0; d < h->D; ++d) units += c[(size_t)d * C_NCOUNT + slot];
    unsigned long long &base = kernel == PIC_KERNEL_COULOMB ? h->coul0 : h->dsmc0;
    // algorithmic bytes.  Coulomb pass: vx, vy, vz read and written for every
    // particle of a cell holding at least two of its species.  Sequential gas
    // scheme: per live slot and part, cell and offset read, vx, vy, vz read
    // and written
    const double R = h->fp64 ? 8.0 : 4.0;
    const double per = kernel == PIC_KERNEL_COULOMB ? 6.0 * R : 4.0 + 7.0 * R;
    if (ms) *ms = h->kms[kernel];
    if (launches) *launches = h->kl[kernel];
    if (bytes) *bytes = (double)(units - base) * per;
    if (reset) {
        h->kms[kernel] = 0.0;
        h->kl[kernel] = 0;
        base = units;
    }
    return PIC_OK;
}

extern "C" void pic_destroy(pic_handle *h)
{
    if (!h) return;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->gexec_cycle) cudaGraphExecDestroy(h->gexec_cycle);
    for (auto &e : h->ev) cudaEventDestroy(e);
    delete h;
}

void o2::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

extern "C" const char *pic_last_error(const pic_handle *h)
{
    if (h) return h->err.c_str();
    return g_err.c_str();
}
