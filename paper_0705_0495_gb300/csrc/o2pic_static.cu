// o2pic_static.cu -- charge deposit and field solve of one discharge from
// particle arrays the caller owns, with no memory allocation anywhere.
//
// Some callers cannot allocate device memory at all: code running inside a
// framework that owns every allocation, code that must not trigger a
// cudaMalloc (which can synchronise the device) in the middle of its own
// work, or code with a fixed memory budget checked up front.  For them the
// charge accumulators live in one file-scope __device__ array of fixed size
// (STATIC_MAX_CELLS + 1 nodes per species), which every GPU that loads this
// library reserves until the process exits.  The caller passes the particle
// arrays and the output arrays; this file never calls cudaMalloc, cudaFree
// or an allocating library routine.
#include <mutex>
#include <string>

#include "../../include/o2pic.h"
#include "o2pic_dev.cuh"
#include "o2pic_launch.h"

namespace {

constexpr int STATIC_MAX_CELLS = 4096;
constexpr int STATIC_NODES = STATIC_MAX_CELLS + 1;
constexpr int STATIC_FIELD_THREADS = 1024;
constexpr double QE_S = 1.602176634e-19;
constexpr double EPS0_S = 8.8541878128e-12;
constexpr int MAX_DEVICES = 64;

// Per-species charge accumulators shared by every call on a device: fixed
// point (weight * 2^FIX_BITS) in the FP32 path, FP64 in the FP64 path; both
// 8 bytes per node.  3 * 4097 * 8 bytes = 98,328 bytes per device.
static __device__ __align__(256) unsigned long long g_static_acc[3 * STATIC_NODES];

std::mutex g_mu;
void *g_acc_ptr[MAX_DEVICES] = {};

__global__ void k_static_deposit_f32(unsigned long long *acc, const int *cell, const float *off, long long n,
                                     int N)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = cell[i];
        if (c < 0 || c >= N) continue;
        // an offset outside [0, 1] (or NaN) is clamped into it, so that the
        // two weights stay within [0, 2^FIX_BITS] and add up to one particle
        const float o = fminf(fmaxf(off[i], 0.0f), 1.0f);
        const unsigned w1 = __float2uint_rn(o * (float)(1 << o2::FIX_BITS));
        const unsigned w0 = (1u << o2::FIX_BITS) - w1;
        atomicAdd(&acc[c], (unsigned long long)w0);
        atomicAdd(&acc[c + 1], (unsigned long long)w1);
    }
}

__global__ void k_static_deposit_f64(double *acc, const int *cell, const double *off, long long n, int N)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = cell[i];
        if (c < 0 || c >= N) continue;
        const double o = fmin(fmax(off[i], 0.0), 1.0);  // clamped as in the FP32 path
        atomicAdd(&acc[c], 1.0 - o);
        atomicAdd(&acc[c + 1], o);
    }
}

// One block: rho from the accumulators, then the Dirichlet problem
// (phi_{i-1} - 2 phi_i + phi_{i+1}) = -rho_i dx^2 / eps0, phi_0 = U(t),
// phi_N = 0, solved exactly by two prefix sums (phi_i = phi_0 + i D0 -
// S2_{i-1}), and E from centred differences with Gauss's law on the half
// cells at the walls.  Sums run sequentially in one thread: N <= 4096.
__global__ void __launch_bounds__(STATIC_FIELD_THREADS)
k_static_field(const unsigned long long *acc, int fp64, int N, double dx, double weight, double phi0,
               double *rho, double *phi, double *E)
{
    extern __shared__ __align__(16) double sx[];  // rho, then S2
    const int tid = threadIdx.x;
    for (int i = tid; i <= N; i += blockDim.x) {
        const double vol = (i == 0 || i == N) ? 0.5 * dx : dx;
        double a[3];
        for (int s = 0; s < 3; ++s) {
            const unsigned long long v = acc[s * STATIC_NODES + i];
            a[s] = fp64 ? __longlong_as_double((long long)v)
                        : (double)(long long)v / (double)(1 << o2::FIX_BITS);
        }
        const double r = QE_S * weight * (a[2] - a[0] - a[1]) / vol;
        rho[i] = r;
        sx[i] = r * dx * dx / EPS0_S;
    }
    __syncthreads();
    if (tid == 0) {
        double s1 = 0.0, s2 = 0.0;
        for (int i = 1; i < N; ++i) {
            s1 += sx[i];
            s2 += s1;
            sx[i] = s2;  // S2_i
        }
        const double D0 = (s2 - phi0) / (double)N;
        phi[0] = phi0;
        for (int i = 1; i < N; ++i) phi[i] = phi0 + (double)i * D0 - (i >= 2 ? sx[i - 1] : 0.0);
        phi[N] = 0.0;
    }
    __syncthreads();
    for (int i = tid; i <= N; i += blockDim.x) {
        double e;
        if (i == 0) e = -(phi[1] - phi[0]) / dx - rho[0] * dx / (2.0 * EPS0_S);
        else if (i == N) e = -(phi[N] - phi[N - 1]) / dx + rho[N] * dx / (2.0 * EPS0_S);
        else e = -(phi[i + 1] - phi[i - 1]) / (2.0 * dx);
        E[i] = e;
    }
}

pic_status static_fail(pic_status s, const std::string &m)
{
    o2::set_last_error(m.c_str());
    return s;
}

} // namespace

extern "C" pic_status pic_field_solve_static(const pic_config *cfg, long long step, const int *const *d_cell,
                                             const void *const *d_off, const long long *n, double *d_rho,
                                             double *d_phi, double *d_E, void *cuda_stream)
{
    if (!cfg || !d_cell || !d_off || !n || !d_rho || !d_phi || !d_E)
        return static_fail(PIC_EINVAL, "pic_field_solve_static: NULL argument");
    const int N = cfg->n_cells;
    if (N < 2 || N > STATIC_MAX_CELLS)
        return static_fail(PIC_EINVAL, "pic_field_solve_static: n_cells must be in [2, 4096] (the size of "
                                       "its fixed scratch array)");
    if (!(cfg->L_m > 0) || !(cfg->dt_s > 0) || !(cfg->weight_m2 >= 0) || step < 0)
        return static_fail(PIC_EINVAL, "pic_field_solve_static: need L > 0, dt > 0, weight >= 0, step >= 0");
    if (cfg->precision != PIC_FP64 && cfg->precision != PIC_FP32_MIXED)
        return static_fail(PIC_EINVAL, "pic_field_solve_static: bad precision");
    for (int s = 0; s < 3; ++s)
        if (n[s] < 0 || (n[s] > 0 && (!d_cell[s] || !d_off[s])))
            return static_fail(PIC_EINVAL, "pic_field_solve_static: bad particle arrays");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return static_fail(PIC_ECUDA, std::string("pic_field_solve_static: cudaGetDevice: ") + cudaGetErrorString(e));
    void *acc = nullptr;
    {
        // set-up, once per device, with that device current: the device
        // address of the scratch array (its host-side name is only a handle)
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_acc_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_acc);
            if (e != cudaSuccess || !p)
                return static_fail(PIC_ECUDA, std::string("pic_field_solve_static: cudaGetSymbolAddress: ") +
                                                  cudaGetErrorString(e));
            g_acc_ptr[dev] = p;
        }
        acc = g_acc_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // the array keeps the previous call's sums: clear it first
    e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 3 * STATIC_NODES, st);
    if (e != cudaSuccess)
        return static_fail(PIC_ECUDA, std::string("pic_field_solve_static: ") + cudaGetErrorString(e));
    const bool fp64 = cfg->precision == PIC_FP64;
    for (int s = 0; s < 3; ++s) {
        if (n[s] == 0) continue;
        const long long blocks = (n[s] + 255) / 256;
        const int grid = (int)(blocks < 4096 ? blocks : 4096);
        unsigned long long *a = static_cast<unsigned long long *>(acc) + (size_t)s * STATIC_NODES;
        if (fp64)
            k_static_deposit_f64<<<grid, 256, 0, st>>>(reinterpret_cast<double *>(a), d_cell[s],
                                                       static_cast<const double *>(d_off[s]), n[s], N);
        else
            k_static_deposit_f32<<<grid, 256, 0, st>>>(a, d_cell[s], static_cast<const float *>(d_off[s]),
                                                       n[s], N);
    }
    const double PI_S = 3.14159265358979323846;
    const double t = (double)step * cfg->dt_s;
    const double phi0 = cfg->U_rf_V * sin(2.0 * PI_S * cfg->f_rf_Hz * t + cfg->rf_phase);
    k_static_field<<<1, STATIC_FIELD_THREADS, sizeof(double) * (N + 1), st>>>(
        static_cast<const unsigned long long *>(acc), fp64 ? 1 : 0, N, cfg->L_m / N, cfg->weight_m2, phi0, d_rho,
        d_phi, d_E);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return static_fail(PIC_ECUDA, std::string("pic_field_solve_static: launch: ") + cudaGetErrorString(e));
    return PIC_OK;
}
