// Allocation-free time step (lelbm_step_noalloc in include/lelbm.h).
//
// Who needs it: callers that must not allocate device memory.  Examples:
//   - an application that owns all device memory through its own pool or a
//     fixed memory budget;
//   - code on a latency-critical path, where cudaFree synchronises the whole
//     device and cudaMalloc can fail or fragment mid-run.
// Such a caller passes the input and output moment buffers it already owns.
// Everything else the step needs (counters, the 1D instance table) lives in
// the file-scope array g_noalloc_scratch below.
//
// The array is a static __device__ variable.  Every GPU on which the library
// is loaded holds its 512 KiB until the process exits.  All calls share it
// and it keeps the last call's contents, so every call clears what must start
// at zero.  Calls whose work overlaps on the GPU (for example on two streams)
// race on it.
//
// In host code the name g_noalloc_scratch is only a host-side stand-in, not a
// device address.  The device address comes from cudaGetSymbolAddress, taken
// once per device with that device current (on the first call there).
// Device code uses the array directly.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/lelbm.h"
#include "lelbm_device.cuh"

namespace lbm {
namespace {

constexpr int kMaxInst = LELBM_NOALLOC_MAX_INSTANCES;
// byte layout of the scratch array
constexpr size_t kStatsOff = 0;
constexpr size_t kLenOff = 1024;                                  // int[kMaxInst]
constexpr size_t kPadOff = kLenOff + sizeof(int) * kMaxInst;      // int[kMaxInst]
constexpr size_t kBlkOff = kPadOff + sizeof(int) * kMaxInst;      // long long[kMaxInst + 1]
constexpr size_t kScratchBytes = kBlkOff + sizeof(long long) * (kMaxInst + 1);
static_assert(sizeof(DevStats) <= kLenOff, "counters overflow their slot");
static_assert(kScratchBytes <= 512 * 1024, "scratch larger than stated");

static __device__ __align__(256) unsigned char g_noalloc_scratch[512 * 1024];

__device__ __forceinline__ DevStats* scratch_stats() {
    return reinterpret_cast<DevStats*>(g_noalloc_scratch + kStatsOff);
}
__device__ __forceinline__ const int* scratch_len() {
    return reinterpret_cast<const int*>(g_noalloc_scratch + kLenOff);
}
__device__ __forceinline__ const int* scratch_pad() {
    return reinterpret_cast<const int*>(g_noalloc_scratch + kPadOff);
}
__device__ __forceinline__ long long* scratch_blk() {
    return reinterpret_cast<long long*>(g_noalloc_scratch + kBlkOff);
}

// Geometry of the step, passed by value.
struct Topo {
    int D;
    long long ncell;
    int NX, NY;          // 2D padded sizes
    int nx, ny, pad;     // 2D interior and pad
    int periodic[2];
    int bc[4];
    int n_inst;          // 1D instances
    int uniform_pad;     // 1D: pad of every instance, or -1 to read the per-instance table
    double inlet[4];
};

// Exclusive prefix sum of the 1D block sizes (pads + interior) into blk[0..n].
__global__ void instance_scan_kernel(int n, int periodic, int uniform_pad) {
    __shared__ long long part[1024];
    const int* len = scratch_len();
    const int* pad = scratch_pad();
    long long* blk = scratch_blk();
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    long long s = 0;
    for (int b = b0; b < n && b < b0 + per; b++)
        s += len[b] + (periodic ? 0 : 2LL * (uniform_pad >= 0 ? uniform_pad : pad[b]));
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int i = 0; i < (int)blockDim.x; i++) {
            const long long v = part[i];
            part[i] = acc;
            acc += v;
        }
    }
    __syncthreads();
    long long acc = part[threadIdx.x];
    for (int b = b0; b < n && b < b0 + per; b++) {
        blk[b] = acc;
        acc += len[b] + (periodic ? 0 : 2LL * (uniform_pad >= 0 ? uniform_pad : pad[b]));
    }
    if (b0 < n && b0 + per >= n) blk[n] = acc;
}

__device__ __forceinline__ int find_instance(const long long* blk, int n, long long cell) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk[mid] <= cell)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <int D>
__global__ void __launch_bounds__(128) noalloc_cell_kernel(Model m, Topo t, const double* __restrict__ Min,
                                                           double* Mout) {
    constexpr int NM = Dim<D>::NM, NF = Dim<D>::NF, NG = Dim<D>::NG;
    DevStats* stats = scratch_stats();
    const long long* blk = scratch_blk();
    const int* len = scratch_len();
    const int* pads = scratch_pad();
    __shared__ unsigned long long s_hist[64];
    __shared__ unsigned long long s_cells, s_feq, s_fmx, s_q, s_dmax, s_pf, s_pg, s_pm;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) s_hist[i] = 0;
    if (threadIdx.x == 0) s_cells = s_feq = s_fmx = s_q = s_dmax = s_pf = s_pg = s_pm = 0;
    __syncthreads();

    unsigned long long my_cells = 0, my_pf = 0, my_pg = 0, my_q = 0, my_pts = 0;
    double my_dmax = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < t.ncell; cell += stride) {
        // where this cell's moments come from (Sec. III.A fill, done on the fly); the same
        // rules as fill_pads_kernel and the pad-source lists the handle builds at create
        long long src = cell;
        bool inflow = false;
        long long lo = 0;
        int n = 0, ix = 0, iy = 0;
        if constexpr (D == 1) {
            const int b = find_instance(blk, t.n_inst, cell);
            const int p = t.periodic[0] ? 0 : (t.uniform_pad >= 0 ? t.uniform_pad : pads[b]);
            n = len[b];
            lo = blk[b] + p;
            if (cell < lo) {
                inflow = t.bc[0] == LELBM_BC_INFLOW;
                src = lo;
            } else if (cell >= lo + n) {
                inflow = t.bc[1] == LELBM_BC_INFLOW;
                src = lo + n - 1;
            }
        } else {
            iy = (int)(cell / t.NX);
            ix = (int)(cell - (long long)iy * t.NX);
            const int px = t.periodic[0] ? 0 : t.pad, py = t.periodic[1] ? 0 : t.pad;
            const bool inx = ix >= px && ix < px + t.nx, iny = iy >= py && iy < py + t.ny;
            if (!(inx && iny)) {
                inflow = (ix < px && t.bc[0] == LELBM_BC_INFLOW) || (ix >= px + t.nx && t.bc[1] == LELBM_BC_INFLOW) ||
                         (iy < py && t.bc[2] == LELBM_BC_INFLOW) || (iy >= py + t.ny && t.bc[3] == LELBM_BC_INFLOW);
                const int sx = ix < px ? px : (ix >= px + t.nx ? px + t.nx - 1 : ix);
                const int sy = iy < py ? py : (iy >= py + t.ny ? py + t.ny - 1 : iy);
                src = (long long)sy * t.NX + sx;
            }
        }
        double M[NM];
        if (inflow) {
            const double uin[2] = {t.inlet[1], t.inlet[2]};
            eq_moments<D>(m.K, t.inlet[0], uin, t.inlet[3], M);
        } else {
#pragma unroll
            for (int i = 0; i < NM; i++) M[i] = Min[i * t.ncell + src];
        }
        CellState<D> c;
        collide<D>(M, m, c);  // as prepare_cell (lelbm_step.cuh) on the FP64 path
        if (!c.ok) {
            atomicAdd(&s_fmx, 1ull);
            atomicMin(&stats->first_fail, (unsigned long long)cell);
            continue;
        }
        my_cells++;
        Stencil<D> st;
        st.init(c, m);
        const bool has_g = m.K > 0.0;
        double lf[NF], lg[NG];
        maxwell_start<D, NF>(c.RT, lf);
        int sf = epr_newton<D, true>(c, st, c.cf, lf, m, my_pf);
        int sg = 0;
        if (has_g) {
            maxwell_start<D, NG>(c.RT, lg);
            sg = epr_newton<D, false>(c, st, c.cg, lg, m, my_pg);
        } else {
#pragma unroll
            for (int j = 0; j < NG; j++) lg[j] = 0.0;
        }
        if (sf >= 0 && sg >= 0) {
            atomicAdd(&s_hist[sf < 63 ? sf : 63], 1ull);
            if (has_g) atomicAdd(&s_hist[sg < 63 ? sg : 63], 1ull);
        } else {
            // the fallback chain of fp64_tail (lelbm_step.cuh): equilibrium constraints, then
            // normalised Maxwellian weights; a change there must be made here too
            double ef[NF], eg[NG];
#pragma unroll
            for (int j = 0; j < NF; j++) ef[j] = 0.0;
#pragma unroll
            for (int j = 0; j < NG; j++) eg[j] = 0.0;
            ef[0] = eg[0] = 1.0;
            int jj = 1 + D;
#pragma unroll
            for (int a = 0; a < D; a++)
#pragma unroll
                for (int b = a; b < D; b++) {
                    ef[jj] = eg[jj] = (a == b) ? 1.0 : 0.0;
                    jj++;
                }
            maxwell_start<D, NF>(c.RT, lf);
            sf = epr_newton<D, true>(c, st, ef, lf, m, my_pf);
            sg = 0;
            if (has_g) {
                maxwell_start<D, NG>(c.RT, lg);
                sg = epr_newton<D, false>(c, st, eg, lg, m, my_pg);
            }
            if (sf >= 0 && sg >= 0) {
                atomicAdd(&s_feq, 1ull);
            } else {
                double S = 0.0;
                auto sum = [&](const double* cp, double dC) {
                    double t2 = 0.0;
#pragma unroll
                    for (int a = 0; a < D; a++) {
                        const double tt = (cp[a] - c.u[a]) * c.inv_sig;
                        t2 += tt * tt;
                    }
                    S += dC * exp(-0.5 * t2);
                };
                st.for_each(sum);
#pragma unroll
                for (int j = 0; j < NF; j++) lf[j] = 0.0;
                lf[0] = log(S) - 1.0;
                jj = 1 + D;
#pragma unroll
                for (int a = 0; a < D; a++)
#pragma unroll
                    for (int b = a; b < D; b++) {
                        lf[jj] = (a == b) ? 0.5 : 0.0;
                        jj++;
                    }
#pragma unroll
                for (int j = 0; j < NG; j++) lg[j] = lf[j];
                atomicAdd(&s_fmx, 1ull);
                atomicMin(&stats->first_fail, (unsigned long long)cell);
            }
        }
        // moment streaming (Eq. IIE3) with the landing rules of the padded layout: those of
        // land() (lelbm_land.cuh) and the cloud-in-cell sharing of scatter_cell (lelbm_step.cuh)
        const double mfs = c.rho, mgs = c.rho * m.K * c.RT;
        unsigned long long q = 0;
        double dmax2 = 0.0;
        auto emit = [&](const double* cp, double dC) {
            q++;
            double tt[D];
#pragma unroll
            for (int a = 0; a < D; a++) tt[a] = (cp[a] - c.u[a]) * c.inv_sig;
            double T[NF];
            Basis<D, true>::eval(tt, T);
            double e = 1.0;
#pragma unroll
            for (int j = 0; j < NF; j++) e += lf[j] * T[j];
            const double mf = mfs * dC * exp(-e);
            double mg = 0.0;
            if (has_g) {
                double eg = 1.0;
#pragma unroll
                for (int j = 0; j < NG; j++) eg += lg[j] * T[j];
                mg = mgs * dC * exp(-eg);
            }
            double csq = 0.0;
#pragma unroll
            for (int a = 0; a < D; a++) csq += cp[a] * cp[a];
            dmax2 = fmax(dmax2, csq);
            double dM[NM];
            dM[0] = mf;
#pragma unroll
            for (int a = 0; a < D; a++) dM[1 + a] = cp[a] * mf;
#pragma unroll
            for (int a = 0; a < D; a++)
#pragma unroll
                for (int b = a; b < D; b++) dM[iM2<D>(a, b)] = cp[a] * cp[b] * mf;
#pragma unroll
            for (int gg = 0; gg < D; gg++) dM[iMD<D>(gg)] = csq * cp[gg] * mf;
            dM[iG0<D>()] = mg;
#pragma unroll
            for (int gg = 0; gg < D; gg++) dM[iG1<D>(gg)] = cp[gg] * mg;
            int base[D];
            double w1[D];
#pragma unroll
            for (int a = 0; a < D; a++) {
                const double fl = floor(cp[a]);
                base[a] = (int)fl;
                w1[a] = cp[a] - fl;
            }
            const int ncx = w1[0] > 0.0 ? 2 : 1;
            const int ncy = (D == 2 && w1[D - 1] > 0.0) ? 2 : 1;
            for (int sy = 0; sy < ncy; sy++)
                for (int sx = 0; sx < ncx; sx++) {
                    double w = sx ? w1[0] : 1.0 - w1[0];
                    long long tgt;
                    if constexpr (D == 1) {
                        long long x = cell + base[0] + sx;
                        if (t.periodic[0]) {
                            long long r = (x - lo) % n;
                            if (r < 0) r += n;
                            x = lo + r;
                        } else if (x < lo || x >= lo + n) {
                            continue;
                        }
                        tgt = x;
                    } else {
                        w *= sy ? w1[D - 1] : 1.0 - w1[D - 1];
                        int tx = ix + base[0] + sx, ty = iy + base[D - 1] + sy;
                        if (t.periodic[0]) {
                            tx %= t.nx;
                            if (tx < 0) tx += t.nx;
                        } else if (tx < t.pad || tx >= t.pad + t.nx) {
                            continue;
                        }
                        if (t.periodic[1]) {
                            ty %= t.ny;
                            if (ty < 0) ty += t.ny;
                        } else if (ty < t.pad || ty >= t.pad + t.ny) {
                            continue;
                        }
                        tgt = (long long)ty * t.NX + tx;
                    }
#pragma unroll
                    for (int mm = 0; mm < NM; mm++) atomicAdd(Mout + mm * t.ncell + tgt, w * dM[mm]);
                }
        };
        st.for_each(emit);
        my_q = q > my_q ? q : my_q;
        my_pts += q;
        my_dmax = fmax(my_dmax, sqrt(dmax2));
    }
    atomicAdd(&s_cells, my_cells);
    atomicAdd(&s_pf, my_pf);
    atomicAdd(&s_pg, my_pg);
    atomicAdd(&s_pm, my_pts);
    atomicMax(&s_q, my_q);
    atomicMax(&s_dmax, (unsigned long long)__double_as_longlong(my_dmax));
    __syncthreads();
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&stats->newton_hist[i], s_hist[i]);
    if (threadIdx.x == 0) {
        atomicAdd(&stats->cells, s_cells);
        atomicAdd(&stats->points_f, s_pf);
        atomicAdd(&stats->points_g, s_pg);
        atomicAdd(&stats->points_ms, s_pm);
        if (s_feq) atomicAdd(&stats->fallback_eq, s_feq);
        if (s_fmx) atomicAdd(&stats->fallback_mx, s_fmx);
        atomicMax(&stats->q_max, s_q);
        atomicMax(&stats->disp_max_bits, s_dmax);
    }
}

// Device address of g_noalloc_scratch, looked up once per device.
std::mutex g_addr_mutex;
unsigned char* g_addr[64] = {};

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lelbm_step_noalloc(const lelbm_params* p, const double* m_in, double* m_out, lelbm_stats* stats) {
    if (!p || !m_in || !m_out) return LELBM_E_INVAL;
    if (p->dims != 1 && p->dims != 2) return LELBM_E_INVAL;
    if (p->solid || p->precision != LELBM_FP64 || p->deterministic) return LELBM_E_INVAL;
    if (p->nx < 1 || p->ny < 1 || (p->dims == 1 && p->ny != 1)) return LELBM_E_INVAL;
    if (!(p->K >= 0.0) || !(p->nu_shear >= 0.0) || !(p->prandtl > 0.0) || !(p->tol > 0.0)) return LELBM_E_INVAL;
    if (p->max_newton < 1 || p->max_newton > 60 || p->max_refine < 0 || p->max_refine > 4) return LELBM_E_INVAL;
    for (int a = 0; a < p->dims; a++) {
        const int l = p->bc[2 * a], r = p->bc[2 * a + 1];
        if (l < 0 || l > 2 || r < 0 || r > 2) return LELBM_E_INVAL;
        if ((l == LELBM_BC_PERIODIC) != (r == LELBM_BC_PERIODIC)) return LELBM_E_INVAL;
        if (l != LELBM_BC_PERIODIC && p->dims == 2 && p->pad < 1) return LELBM_E_INVAL;
    }
    const int nb = (p->dims == 1 && p->n_batch > 1) ? p->n_batch : 1;
    if (nb > kMaxInst) return LELBM_E_INVAL;  // beyond the scratch array's capacity
    const bool periodic_x = p->bc[0] == LELBM_BC_PERIODIC;
    if (p->dims == 1 && !periodic_x && !(nb > 1 && p->pads) && p->pad < 1) return LELBM_E_INVAL;
    if (nb > 1 && !p->lengths) return LELBM_E_INVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LELBM_E_CUDA;
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mutex);
        if (!g_addr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess) return LELBM_E_CUDA;
            g_addr[dev] = static_cast<unsigned char*>(ptr);
        }
        base = g_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)p->stream;

    Model m{};
    m.K = p->K;
    m.inv_dk = 1.0 / ((double)p->dims + p->K);
    m.nu_s = p->nu_shear;
    m.nu_b = p->nu_bulk;
    m.Pr = p->prandtl;
    m.limiter = p->limiter;
    m.n_conf = p->n_conform;
    m.r_min = p->r_min;
    m.refine_div = p->refine_div;
    m.refine_rad = p->refine_rad;
    m.max_refine = p->max_refine;
    m.tol = p->tol;
    m.max_iter = p->max_newton;
    set_fp32_params(m);

    Topo t{};
    t.D = p->dims;
    t.periodic[0] = periodic_x;
    t.periodic[1] = p->dims == 2 ? p->bc[2] == LELBM_BC_PERIODIC : 1;
    for (int i = 0; i < 4; i++) {
        t.bc[i] = p->bc[i];
        t.inlet[i] = p->inlet[i];
    }
    t.n_inst = nb;
    long long ncell = 0;
    if (p->dims == 1) {
        // instance lengths and pads go straight from the caller's host arrays into the scratch
        if (nb > 1) {
            if (cudaMemcpyAsync(base + kLenOff, p->lengths, sizeof(int) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return LELBM_E_CUDA;
        } else {
            if (cudaMemcpyAsync(base + kLenOff, &p->nx, sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
                return LELBM_E_CUDA;
        }
        const int* pads_src = (nb > 1 && p->pads) ? p->pads : nullptr;
        if (pads_src) {
            for (int b = 0; b < nb; b++)
                if (!periodic_x && pads_src[b] < 1) return LELBM_E_INVAL;
            if (cudaMemcpyAsync(base + kPadOff, pads_src, sizeof(int) * nb, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return LELBM_E_CUDA;
        }
        t.uniform_pad = pads_src ? -1 : p->pad;
        for (int b = 0; b < nb; b++) {
            const int n = nb > 1 ? p->lengths[b] : p->nx;
            if (n < 1) return LELBM_E_INVAL;
            ncell += n + (periodic_x ? 0 : 2LL * (pads_src ? pads_src[b] : p->pad));
        }
        instance_scan_kernel<<<1, 1024, 0, s>>>(nb, periodic_x ? 1 : 0, t.uniform_pad);
    } else {
        const int px = t.periodic[0] ? 0 : p->pad, py = t.periodic[1] ? 0 : p->pad;
        t.NX = p->nx + 2 * px;
        t.NY = p->ny + 2 * py;
        t.nx = p->nx;
        t.ny = p->ny;
        t.pad = (t.periodic[0] && t.periodic[1]) ? 0 : p->pad;
        ncell = (long long)t.NX * t.NY;
    }
    t.ncell = ncell;

    // counters start at zero (first_fail at its "none" value); the output is accumulated into
    DevStats z;
    std::memset(&z, 0, sizeof z);
    z.first_fail = ~0ull;
    if (cudaMemcpyAsync(base + kStatsOff, &z, sizeof z, cudaMemcpyHostToDevice, s) != cudaSuccess) return LELBM_E_CUDA;
    const int nm = p->dims == 1 ? 6 : 11;
    if (cudaMemsetAsync(m_out, 0, sizeof(double) * nm * ncell, s) != cudaSuccess) return LELBM_E_CUDA;

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long need = (ncell + 127) / 128;
    long long cap = 8LL * (sms > 0 ? sms : 1);
    const int blocks = (int)(need < cap ? need : cap);
    if (p->dims == 1)
        noalloc_cell_kernel<1><<<blocks, 128, 0, s>>>(m, t, m_in, m_out);
    else
        noalloc_cell_kernel<2><<<blocks, 128, 0, s>>>(m, t, m_in, m_out);
    if (cudaGetLastError() != cudaSuccess) return LELBM_E_CUDA;

    if (stats) {
        DevStats d;
        if (cudaMemcpyAsync(&d, base + kStatsOff, sizeof d, cudaMemcpyDeviceToHost, s) != cudaSuccess) return LELBM_E_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return LELBM_E_CUDA;
        std::memset(stats, 0, sizeof *stats);
        stats->steps = 1;
        stats->cells = (long long)d.cells;
        for (int i = 0; i < 64; i++) stats->newton_hist[i] = (long long)d.newton_hist[i];
        stats->fallback_eq = (long long)d.fallback_eq;
        stats->fallback_mx = (long long)d.fallback_mx;
        stats->q_max = (long long)d.q_max;
        double dm;
        std::memcpy(&dm, &d.disp_max_bits, sizeof dm);
        stats->disp_max = dm;
        stats->first_fail_cell = d.first_fail == ~0ull ? -1 : (long long)d.first_fail;
        stats->points_f = (long long)d.points_f;
        stats->points_g = (long long)d.points_g;
        stats->points_ms = (long long)d.points_ms;
        if (d.fallback_mx) return LELBM_E_EPR;
    }
    return LELBM_OK;
}
