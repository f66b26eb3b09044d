// Host side of the C ABI declared in include/lelbm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/lelbm.h"
#include "lelbm_internal.h"

using namespace lbm;

struct lelbm {
    lelbm_params p;
    int D = 1, nmom = 6;
    int NX = 0, NY = 1, NZ = 1;
    long long ncell = 0;
    Model model{};
    Geometry geo{};
    Geometry3 geo3{};
    // host copies of the layout
    std::vector<long long> inst_lo_h;
    std::vector<int> inst_n_h;
    // device memory
    double* M[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t* d_type = nullptr;
    uint8_t* d_wall_dist = nullptr;  // 2D with solids: Chebyshev distance to a solid cell
    uint8_t* d_noslip = nullptr;     // 2D with no-slip walls: their cells
    int* d_inst = nullptr;
    long long* d_inst_lo = nullptr;
    int* d_inst_n = nullptr;
    long long* d_pad_cell = nullptr;
    long long* d_pad_src = nullptr;
    long long npad = 0;
    DevStats* d_stats = nullptr;
    unsigned long long* d_work = nullptr;  // work counter of the cell-update kernel
    // persistent 1D batch
    int* d_order[2] = {nullptr, nullptr};  // batch order, longest first
    long long* d_inst_first = nullptr;     // first cell of each instance block (pads included)
    int* d_inst_pad = nullptr;
    int* d_steps_left = nullptr;
    bool budgets = false;
    lelbm_tuning tuning{128, 0, 0, 0.0};
    __nv_bfloat16* d_mlp_w = nullptr;  // learned warm start: BF16 weights
    float* d_mlp_nrm = nullptr;        // and normalisation
    float* d_lam = nullptr;            // stored warm start (lelbm_set_warmstart)
    float* d_mlp_start = nullptr;      // learned start of the current step (cell-update path)
    double* d_det_lam = nullptr;       // deterministic streaming: per-cell multipliers
    int* d_det_halo = nullptr;         // and the reach of the step's velocity sets
    cudaGraphExec_t graph = nullptr;  // captured lelbm_run_batch launch
    int graph_n = -1, graph_cur = -1;
    bool graph_budgets = false;
    lelbm_tuning graph_tuning{0, 0, 0, 0.0};
    long long steps = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int blocks = 0;
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
    double timed_ms = 0.0;
    long long timed_launches = 0;
    std::string err;
};

static thread_local std::string g_create_err;

static int fail(lelbm_t h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_create_err = buf;
    return code;
}

#define CUDA_TRY(h, call)                                                                             \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return fail((h), LELBM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" void lelbm_abi_sizes(long long* params_size, long long* stats_size) {
    if (params_size) *params_size = (long long)sizeof(lelbm_params);
    if (stats_size) *stats_size = (long long)sizeof(lelbm_stats);
}

extern "C" void lelbm_default_params(lelbm_params* p) {
    std::memset(p, 0, sizeof *p);
    p->dims = 1;
    p->nx = 1;
    p->ny = 1;
    p->nz = 1;
    p->bc[0] = p->bc[1] = p->bc[2] = p->bc[3] = LELBM_BC_PERIODIC;
    p->bc_z[0] = p->bc_z[1] = LELBM_BC_PERIODIC;
    p->inlet[0] = 1.0;
    p->inlet[3] = 1.0;
    p->K = 0.0;
    p->nu_shear = 1e-3;
    p->nu_bulk = -1.0;
    p->prandtl = 1.0;
    p->limiter = 1;
    p->n_conform = 4.0;
    p->r_min = 2.0;
    p->refine_div = 3.0;
    p->refine_rad = 3.0;
    p->max_refine = 4;
    p->tol = 1e-12;
    p->max_newton = 50;
    p->precision = LELBM_FP64;
}

static int validate(const lelbm_params* p) {
    if (!p) return fail(nullptr, LELBM_E_INVAL, "params is NULL");
    if (p->dims < 1 || p->dims > 3) return fail(nullptr, LELBM_E_INVAL, "dims must be 1, 2 or 3");
    if (p->nx < 1 || p->ny < 1) return fail(nullptr, LELBM_E_INVAL, "nx, ny must be >= 1");
    if (p->dims == 1 && p->ny != 1) return fail(nullptr, LELBM_E_INVAL, "ny must be 1 in 1D");
    if (p->dims >= 2 && p->n_batch > 1) return fail(nullptr, LELBM_E_INVAL, "batches are 1D only");
    if (p->dims == 2 && p->solid && p->precision != LELBM_FP64) {
        const int qx = p->bc[0] == LELBM_BC_PERIODIC ? 0 : p->pad, qy = p->bc[2] == LELBM_BC_PERIODIC ? 0 : p->pad;
        const long long nc = (long long)(p->nx + 2 * qx) * (p->ny + 2 * qy);
        for (long long i = 0; i < nc; i++)
            if (p->solid[i] >= 2) return fail(nullptr, LELBM_E_INVAL, "no-slip walls need the FP64 path");
    }
    if (!std::isfinite(p->wall_u[0]) || !std::isfinite(p->wall_u[1]))
        return fail(nullptr, LELBM_E_INVAL, "wall_u must be finite");
    if (p->deterministic && (p->dims != 2 || p->precision != LELBM_FP64 || p->solid))
        return fail(nullptr, LELBM_E_INVAL, "deterministic streaming needs a 2D FP64 grid without solid cells");
    if (p->dims == 3) {
        if (p->nz < 1) return fail(nullptr, LELBM_E_INVAL, "nz must be >= 1 in 3D");
        if (p->precision != LELBM_FP64) return fail(nullptr, LELBM_E_INVAL, "3D runs the FP64 path only");
        if (p->solid) return fail(nullptr, LELBM_E_INVAL, "3D has no solid cells");
        if (!std::isfinite(p->inlet_uz)) return fail(nullptr, LELBM_E_INVAL, "inlet_uz must be finite");
    }
    for (int a = 0; a < p->dims; a++) {
        const int l = a < 2 ? p->bc[2 * a] : p->bc_z[0], r = a < 2 ? p->bc[2 * a + 1] : p->bc_z[1];
        if (l < 0 || l > 2 || r < 0 || r > 2) return fail(nullptr, LELBM_E_INVAL, "bad bc kind");
        if ((l == LELBM_BC_PERIODIC) != (r == LELBM_BC_PERIODIC))
            return fail(nullptr, LELBM_E_INVAL, "periodic must be set on both sides of axis %d", a);
        if (l != LELBM_BC_PERIODIC && p->pad < 1)
            return fail(nullptr, LELBM_E_INVAL, "non-periodic axis %d needs pad >= 1", a);
    }
    if (!(p->K >= 0.0) || !std::isfinite(p->K)) return fail(nullptr, LELBM_E_INVAL, "K must be >= 0");
    if (!(p->nu_shear >= 0.0)) return fail(nullptr, LELBM_E_INVAL, "nu_shear must be >= 0");
    if (!(p->prandtl > 0.0)) return fail(nullptr, LELBM_E_INVAL, "prandtl must be > 0");
    if (!(p->n_conform > 0.0) || !(p->r_min >= 1.0)) return fail(nullptr, LELBM_E_INVAL, "bad stencil radius");
    if (!(p->refine_div > 0.0) || !(p->refine_rad > 0.0)) return fail(nullptr, LELBM_E_INVAL, "bad refinement");
    if (p->max_refine < 0 || p->max_refine > 4) return fail(nullptr, LELBM_E_INVAL, "max_refine must be 0..4");
    if (!(p->tol > 0.0)) return fail(nullptr, LELBM_E_INVAL, "tol must be > 0");
    if (p->max_newton < 1 || p->max_newton > 60) return fail(nullptr, LELBM_E_INVAL, "max_newton must be 1..60");
    if (p->precision != LELBM_FP64 && p->precision != LELBM_MIXED && p->precision != LELBM_FP32)
        return fail(nullptr, LELBM_E_INVAL, "unknown precision");
    if (p->dims == 1 && p->n_batch > 1 && p->lengths)
        for (int b = 0; b < p->n_batch; b++)
            if (p->lengths[b] < 1) return fail(nullptr, LELBM_E_INVAL, "lengths[%d] < 1", b);
    if (p->dims == 1 && p->n_batch > 1 && p->pads && p->bc[0] != LELBM_BC_PERIODIC)
        for (int b = 0; b < p->n_batch; b++)
            if (p->pads[b] < 1) return fail(nullptr, LELBM_E_INVAL, "pads[%d] < 1", b);
    if (p->dims == 2 && p->bc[0] == LELBM_BC_PERIODIC && p->bc[2] == LELBM_BC_PERIODIC && p->pad != 0)
        return fail(nullptr, LELBM_E_INVAL, "pad must be 0 on a fully periodic grid");
    if (p->dims == 3 && p->bc[0] == LELBM_BC_PERIODIC && p->bc[2] == LELBM_BC_PERIODIC &&
        p->bc_z[0] == LELBM_BC_PERIODIC && p->pad != 0)
        return fail(nullptr, LELBM_E_INVAL, "pad must be 0 on a fully periodic grid");
    const double* in = p->inlet;
    bool any_in = false;
    for (int s = 0; s < 2 * p->dims; s++) any_in = any_in || (s < 4 ? p->bc[s] : p->bc_z[s - 4]) == LELBM_BC_INFLOW;
    if (any_in && !(in[0] > 0.0 && in[3] > 0.0)) return fail(nullptr, LELBM_E_INVAL, "inflow state needs rho, RT > 0");
    return LELBM_OK;
}

static void free_all(lelbm* h) {
    for (auto& e : h->ev_used) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (auto& e : h->ev_free) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    cudaFree(h->M[0]);
    cudaFree(h->M[1]);
    cudaFree(h->d_type);
    cudaFree(h->d_wall_dist);
    cudaFree(h->d_noslip);
    cudaFree(h->d_inst);
    cudaFree(h->d_inst_lo);
    cudaFree(h->d_inst_n);
    cudaFree(h->d_pad_cell);
    cudaFree(h->d_pad_src);
    cudaFree(h->d_stats);
    cudaFree(h->d_work);
    cudaFree(h->d_order[0]);
    cudaFree(h->d_order[1]);
    cudaFree(h->d_inst_first);
    cudaFree(h->d_inst_pad);
    cudaFree(h->d_steps_left);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    cudaFree(h->d_mlp_w);
    cudaFree(h->d_mlp_nrm);
    cudaFree(h->d_lam);
    cudaFree(h->d_mlp_start);
    cudaFree(h->d_det_lam);
    cudaFree(h->d_det_halo);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

// Chebyshev distance (in cells, capped at 255) from every padded cell to the nearest
// solid cell: a breadth-first search over the 8-neighbourhood from all solid cells,
// wrapping periodic axes.  The streaming pass traces paths past solid faces only in
// cells whose populations can reach that far.
static std::vector<uint8_t> wall_distance(const std::vector<uint8_t>& type, int NX, int NY, bool per_x,
                                          bool per_y) {
    const long long n = (long long)NX * NY;
    std::vector<uint8_t> dist(n, 255);
    std::vector<long long> frontier, next;
    for (long long i = 0; i < n; i++)
        if (type[i] == CELL_SOLID) {
            dist[i] = 0;
            frontier.push_back(i);
        }
    for (int d = 1; d < 255 && !frontier.empty(); d++) {
        next.clear();
        for (long long c : frontier) {
            const int y = (int)(c / NX), x = (int)(c - (long long)y * NX);
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int tx = x + dx, ty = y + dy;
                    if (per_x) tx = (tx + NX) % NX;
                    if (per_y) ty = (ty + NY) % NY;
                    if (tx < 0 || tx >= NX || ty < 0 || ty >= NY) continue;
                    const long long t = (long long)ty * NX + tx;
                    if (dist[t] == 255) {
                        dist[t] = (uint8_t)d;
                        next.push_back(t);
                    }
                }
        }
        frontier.swap(next);
    }
    return dist;
}

template <class T>
static int upload(lelbm* h, T** dst, const std::vector<T>& src) {
    if (src.empty()) return LELBM_OK;
    CUDA_TRY(h, cudaMalloc((void**)dst, sizeof(T) * src.size()));
    CUDA_TRY(h, cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return LELBM_OK;
}

static int reset_stats_dev(lelbm* h) {
    DevStats z;
    std::memset(&z, 0, sizeof z);
    z.first_fail = ~0ull;
    CUDA_TRY(h, cudaMemcpyAsync(h->d_stats, &z, sizeof z, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->steps = 0;
    h->timed_ms = 0.0;
    h->timed_launches = 0;
    return LELBM_OK;
}

extern "C" int lelbm_create(lelbm_t* out, const lelbm_params* p) {
    g_create_err.clear();
    if (!out) return fail(nullptr, LELBM_E_INVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev < 1)
        return fail(nullptr, LELBM_E_CUDA, "no CUDA device: %s", cudaGetErrorString(ce));

    lelbm* h = new (std::nothrow) lelbm();
    if (!h) return fail(nullptr, LELBM_E_NOMEM, "host allocation failed");
    h->p = *p;
    h->p.lengths = nullptr;
    h->p.pads = nullptr;
    h->p.solid = nullptr;
    const int D = p->dims;
    h->D = D;
    h->nmom = D == 1 ? 6 : (D == 2 ? 11 : 17);
    cudaGetDevice(&h->device);
    if (p->stream) {
        h->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(nullptr, LELBM_E_CUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    Model& m = h->model;
    m.lam_store = nullptr;
    m.K = p->K;
    m.inv_dk = 1.0 / ((double)D + p->K);
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

    Geometry& g = h->geo;
    g.D = D;
    g.periodic[0] = p->bc[0] == LELBM_BC_PERIODIC;
    g.periodic[1] = D == 2 ? p->bc[2] == LELBM_BC_PERIODIC : 1;
    std::vector<uint8_t> type;
    std::vector<uint8_t> noslip;  // 2D: 1 on no-slip wall cells (solid byte 2)
    std::vector<long long> pad_cell, pad_src;
    if (D == 1) {
        const int nb = p->n_batch > 1 ? p->n_batch : 1;
        std::vector<int> inst;
        long long off = 0;
        int pad = 0;
        for (int b = 0; b < nb; b++) {
            const int n = (p->n_batch > 1 && p->lengths) ? p->lengths[b] : p->nx;
            pad = g.periodic[0] ? 0 : ((p->n_batch > 1 && p->pads) ? p->pads[b] : p->pad);
            h->inst_lo_h.push_back(off + pad);
            h->inst_n_h.push_back(n);
            for (int i = 0; i < n + 2 * pad; i++) {
                const long long cell = off + i;
                inst.push_back(b);
                if (i < pad || i >= pad + n) {
                    const bool left = i < pad;
                    const bool inflow = p->bc[left ? 0 : 1] == LELBM_BC_INFLOW;
                    type.push_back(inflow ? CELL_PAD_IN : CELL_PAD_OUT);
                    pad_cell.push_back(cell);
                    pad_src.push_back(inflow ? -1 : (left ? off + pad : off + pad + n - 1));
                } else {
                    type.push_back(CELL_FLUID);
                }
            }
            off += n + 2 * pad;
        }
        h->ncell = off;
        h->NX = (int)std::min<long long>(off, 0x7fffffff);
        h->NY = 1;
        g.nx = p->nx;
        g.ny = 1;
        g.pad = pad;
        g.n_inst = nb;
        rc = upload(h, &h->d_inst, inst);
        if (!rc) rc = upload(h, &h->d_inst_lo, h->inst_lo_h);
        if (!rc) rc = upload(h, &h->d_inst_n, h->inst_n_h);
        std::vector<long long> firsts;
        std::vector<int> pads_v, ord0(nb), ord1(nb);
        for (int b = 0; b < nb; b++) {
            const int pb = g.periodic[0] ? 0 : ((p->n_batch > 1 && p->pads) ? p->pads[b] : p->pad);
            pads_v.push_back(pb);
            firsts.push_back(h->inst_lo_h[b] - pb);
            ord0[b] = ord1[b] = b;
        }
        std::stable_sort(ord1.begin(), ord1.end(),
                         [&](int x, int y) { return h->inst_n_h[x] > h->inst_n_h[y]; });
        if (!rc) rc = upload(h, &h->d_inst_first, firsts);
        if (!rc) rc = upload(h, &h->d_inst_pad, pads_v);
        if (!rc) rc = upload(h, &h->d_order[0], ord0);
        if (!rc) rc = upload(h, &h->d_order[1], ord1);
        if (rc) {
            std::string e = h->err;
            free_all(h);
            delete h;
            return fail(nullptr, rc, "%s", e.c_str());
        }
    } else if (D == 3) {
        Geometry3& g3 = h->geo3;
        g3.periodic[0] = p->bc[0] == LELBM_BC_PERIODIC;
        g3.periodic[1] = p->bc[2] == LELBM_BC_PERIODIC;
        g3.periodic[2] = p->bc_z[0] == LELBM_BC_PERIODIC;
        const int px = g3.periodic[0] ? 0 : p->pad, py = g3.periodic[1] ? 0 : p->pad;
        const int pz = g3.periodic[2] ? 0 : p->pad;
        const int NX = p->nx + 2 * px, NY = p->ny + 2 * py, NZ = p->nz + 2 * pz;
        h->NX = NX;
        h->NY = NY;
        h->NZ = NZ;
        h->ncell = (long long)NX * NY * NZ;
        g3.NX = NX;
        g3.NY = NY;
        g3.NZ = NZ;
        g3.ncell = h->ncell;
        g3.nx = p->nx;
        g3.ny = p->ny;
        g3.nz = p->nz;
        g3.px = px;
        g3.py = py;
        g3.pz = pz;
        g.nx = p->nx;
        g.ny = p->ny;
        g.n_inst = 1;
        type.resize(h->ncell);
        const int bcs[6] = {p->bc[0], p->bc[1], p->bc[2], p->bc[3], p->bc_z[0], p->bc_z[1]};
        for (int iz = 0; iz < NZ; iz++)
            for (int iy = 0; iy < NY; iy++)
                for (int ix = 0; ix < NX; ix++) {
                    const long long cell = ((long long)iz * NY + iy) * NX + ix;
                    const bool inx = ix >= px && ix < px + p->nx;
                    const bool iny = iy >= py && iy < py + p->ny;
                    const bool inz = iz >= pz && iz < pz + p->nz;
                    if (inx && iny && inz) {
                        type[cell] = CELL_FLUID;
                        continue;
                    }
                    // Sec. III.A: an inflow side wins at edges and corners
                    bool inflow = false;
                    if (ix < px && bcs[0] == LELBM_BC_INFLOW) inflow = true;
                    if (ix >= px + p->nx && bcs[1] == LELBM_BC_INFLOW) inflow = true;
                    if (iy < py && bcs[2] == LELBM_BC_INFLOW) inflow = true;
                    if (iy >= py + p->ny && bcs[3] == LELBM_BC_INFLOW) inflow = true;
                    if (iz < pz && bcs[4] == LELBM_BC_INFLOW) inflow = true;
                    if (iz >= pz + p->nz && bcs[5] == LELBM_BC_INFLOW) inflow = true;
                    type[cell] = inflow ? CELL_PAD_IN : CELL_PAD_OUT;
                    pad_cell.push_back(cell);
                    if (inflow) {
                        pad_src.push_back(-1);
                    } else {
                        const int sx = std::min(std::max(ix, px), px + p->nx - 1);
                        const int sy = std::min(std::max(iy, py), py + p->ny - 1);
                        const int sz = std::min(std::max(iz, pz), pz + p->nz - 1);
                        pad_src.push_back(((long long)sz * NY + sy) * NX + sx);
                    }
                }
        g.pad = (g3.periodic[0] && g3.periodic[1] && g3.periodic[2]) ? 0 : p->pad;
    } else {
        const int px = g.periodic[0] ? 0 : p->pad;
        const int py = g.periodic[1] ? 0 : p->pad;
        // one pad width for all non-periodic sides; periodic axes have none
        const int NX = p->nx + 2 * px, NY = p->ny + 2 * py;
        h->NX = NX;
        h->NY = NY;
        h->ncell = (long long)NX * NY;
        g.nx = p->nx;
        g.ny = p->ny;
        g.n_inst = 1;
        type.resize(h->ncell);
        noslip.assign(h->ncell, 0);
        for (int iy = 0; iy < NY; iy++)
            for (int ix = 0; ix < NX; ix++) {
                const long long cell = (long long)iy * NX + ix;
                const bool inx = ix >= px && ix < px + p->nx;
                const bool iny = iy >= py && iy < py + p->ny;
                if (inx && iny) {
                    type[cell] = (p->solid && p->solid[cell]) ? CELL_SOLID : CELL_FLUID;
                    noslip[cell] = (p->solid && (p->solid[cell] == 2 || p->solid[cell] == 3)) ? p->solid[cell] - 1 : 0;
                    continue;
                }
                bool inflow = false;
                if (ix < px && p->bc[0] == LELBM_BC_INFLOW) inflow = true;
                if (ix >= px + p->nx && p->bc[1] == LELBM_BC_INFLOW) inflow = true;
                if (iy < py && p->bc[2] == LELBM_BC_INFLOW) inflow = true;
                if (iy >= py + p->ny && p->bc[3] == LELBM_BC_INFLOW) inflow = true;
                if (inflow) {
                    type[cell] = CELL_PAD_IN;
                    pad_cell.push_back(cell);
                    pad_src.push_back(-1);
                } else {
                    const int sx = std::min(std::max(ix, px), px + p->nx - 1);
                    const int sy = std::min(std::max(iy, py), py + p->ny - 1);
                    const long long src = (long long)sy * NX + sx;
                    if (p->solid && p->solid[src]) {
                        // the wall continues through an outflow pad whose nearest interior
                        // cell is solid (instead of the pad copying an empty state)
                        type[cell] = CELL_SOLID;
                        noslip[cell] = (p->solid[src] == 2 || p->solid[src] == 3) ? p->solid[src] - 1 : 0;
                        continue;
                    }
                    type[cell] = CELL_PAD_OUT;
                    pad_cell.push_back(cell);
                    pad_src.push_back(src);
                }
            }
        // interior offset of every non-periodic axis (periodic axes have no pads)
        g.pad = (g.periodic[0] && g.periodic[1]) ? 0 : p->pad;
    }
    g.NX = h->NX;
    g.NY = h->NY;
    g.ncell = h->ncell;
    g.wall_u[0] = p->wall_u[0];
    g.wall_u[1] = p->wall_u[1];
    g.inst_of_cell = h->d_inst;
    g.inst_lo = h->d_inst_lo;
    g.inst_n = h->d_inst_n;
    h->npad = (long long)pad_cell.size();

    const size_t bytes = sizeof(double) * (size_t)h->nmom * (size_t)h->ncell;
    cudaError_t e1 = cudaMalloc((void**)&h->M[0], bytes);
    cudaError_t e2 = cudaMalloc((void**)&h->M[1], bytes);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        free_all(h);
        delete h;
        return fail(nullptr, LELBM_E_NOMEM, "cudaMalloc of %zu bytes failed", 2 * bytes);
    }
    rc = upload(h, &h->d_type, type);
    if (!rc && D == 2 && std::find(type.begin(), type.end(), (uint8_t)CELL_SOLID) != type.end()) {
        rc = upload(h, &h->d_wall_dist, wall_distance(type, h->NX, h->NY, g.periodic[0], g.periodic[1]));
        g.wall_dist = h->d_wall_dist;
        if (!rc && std::any_of(noslip.begin(), noslip.end(), [](uint8_t v) { return v != 0; })) {
            rc = upload(h, &h->d_noslip, noslip);
            g.noslip = h->d_noslip;
        }
    }
    if (!rc) rc = upload(h, &h->d_pad_cell, pad_cell);
    if (!rc) rc = upload(h, &h->d_pad_src, pad_src);
    if (!rc && cudaMalloc((void**)&h->d_stats, sizeof(DevStats)) != cudaSuccess) rc = LELBM_E_NOMEM;
    if (!rc && cudaMalloc((void**)&h->d_work, sizeof(unsigned long long)) != cudaSuccess) rc = LELBM_E_NOMEM;
    if (!rc && (cudaMemset(h->M[0], 0, bytes) != cudaSuccess || cudaMemset(h->M[1], 0, bytes) != cudaSuccess))
        rc = LELBM_E_CUDA;
    if (!rc && p->deterministic) {
        if (cudaMalloc((void**)&h->d_det_lam, sizeof(double) * 16 * (size_t)h->ncell) != cudaSuccess ||
            cudaMalloc((void**)&h->d_det_halo, sizeof(int)) != cudaSuccess)
            rc = LELBM_E_NOMEM;
    }
    if (!rc) rc = reset_stats_dev(h);
    if (rc) {
        std::string e = h->err;
        free_all(h);
        delete h;
        return fail(nullptr, rc, "%s", e.empty() ? "device set-up failed" : e.c_str());
    }
    h->blocks = D == 3 ? cell3d_blocks(h->device) : cell_update_blocks(D, p->precision, h->device);
    *out = h;
    return LELBM_OK;
}

extern "C" void lelbm_destroy(lelbm_t h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

extern "C" int lelbm_layout(lelbm_t h, long long* n_cells, int* n_mom, int* NX, int* NY) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (n_cells) *n_cells = h->ncell;
    if (n_mom) *n_mom = h->nmom;
    if (NX) *NX = h->NX;
    if (NY) *NY = h->NY;
    return LELBM_OK;
}

extern "C" int lelbm_instance(lelbm_t h, int b, long long* first, int* length) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (h->D != 1) {
        if (b != 0) return fail(h, LELBM_E_INVAL, "2D grids have one instance");
        if (first) *first = 0;
        if (length) *length = (int)h->ncell;
        return LELBM_OK;
    }
    if (b < 0 || b >= (int)h->inst_lo_h.size()) return fail(h, LELBM_E_INVAL, "instance %d out of range", b);
    if (first) *first = h->inst_lo_h[b];
    if (length) *length = h->inst_n_h[b];
    return LELBM_OK;
}

extern "C" int lelbm_set_state(lelbm_t h, const double* rho, const double* u, const double* RT) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!rho || !u || !RT) return fail(h, LELBM_E_INVAL, "NULL field");
    const long long n = h->ncell;
    // host-side validation of the interior fluid cells
    std::vector<uint8_t> type(n);
    CUDA_TRY(h, cudaMemcpy(type.data(), h->d_type, n, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < n; i++) {
        if (type[i] != CELL_FLUID) continue;
        bool ok = rho[i] > 0.0 && RT[i] > 0.0 && std::isfinite(rho[i]) && std::isfinite(RT[i]);
        for (int a = 0; a < h->D; a++) ok = ok && std::isfinite(u[a * n + i]);
        if (!ok) return fail(h, LELBM_E_STATE, "non-physical state at cell %lld", i);
    }
    double *dr = nullptr, *du = nullptr, *dT = nullptr;
    if (cudaMalloc((void**)&dr, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc((void**)&du, sizeof(double) * n * h->D) != cudaSuccess ||
        cudaMalloc((void**)&dT, sizeof(double) * n) != cudaSuccess) {
        cudaFree(dr);
        cudaFree(du);
        cudaFree(dT);
        cudaGetLastError();  // clear the allocation error so later launch checks do not see it
        return fail(h, LELBM_E_NOMEM, "set_state: device allocation of the fields failed");
    }
    cudaMemcpyAsync(dr, rho, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(du, u, sizeof(double) * n * h->D, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dT, RT, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
    launch_eq_state(h->D, h->model.K, h->d_type, dr, du, dT, h->M[h->cur], n, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    cudaFree(dr);
    cudaFree(du);
    cudaFree(dT);
    if (e != cudaSuccess) return fail(h, LELBM_E_CUDA, "set_state: %s", cudaGetErrorString(e));
    return LELBM_OK;
}

extern "C" int lelbm_set_moments(lelbm_t h, const double* m) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!m) return fail(h, LELBM_E_INVAL, "NULL moments");
    const size_t bytes = sizeof(double) * (size_t)h->nmom * (size_t)h->ncell;
    CUDA_TRY(h, cudaMemcpyAsync(h->M[h->cur], m, bytes, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LELBM_OK;
}

extern "C" int lelbm_set_moments_device(lelbm_t h, const double* m_dev) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!m_dev) return fail(h, LELBM_E_INVAL, "NULL moments");
    const size_t bytes = sizeof(double) * (size_t)h->nmom * (size_t)h->ncell;
    CUDA_TRY(h, cudaMemcpyAsync(h->M[h->cur], m_dev, bytes, cudaMemcpyDeviceToDevice, h->stream));
    return LELBM_OK;
}

static int take_events(lelbm* h, std::pair<cudaEvent_t, cudaEvent_t>* ev) {
    if (!h->ev_free.empty()) {
        *ev = h->ev_free.back();
        h->ev_free.pop_back();
        return LELBM_OK;
    }
    CUDA_TRY(h, cudaEventCreate(&ev->first));
    CUDA_TRY(h, cudaEventCreate(&ev->second));
    return LELBM_OK;
}

static int collect_timing(lelbm* h) {
    for (auto& e : h->ev_used) {
        float ms = 0.f;
        CUDA_TRY(h, cudaEventElapsedTime(&ms, e.first, e.second));
        h->timed_ms += ms;
        h->timed_launches++;
        h->ev_free.push_back(e);
    }
    h->ev_used.clear();
    return LELBM_OK;
}

extern "C" int lelbm_step(lelbm_t h, int n) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (n < 0) return fail(h, LELBM_E_INVAL, "n must be >= 0");
    const size_t bytes = sizeof(double) * (size_t)h->nmom * (size_t)h->ncell;
    for (int s = 0; s < n; s++) {
        double* Min = h->M[h->cur];
        double* Mout = h->M[1 - h->cur];
        if (h->D == 3) {
            const double in5[5] = {h->p.inlet[0], h->p.inlet[1], h->p.inlet[2], h->p.inlet_uz, h->p.inlet[3]};
            launch_fill_pads3(h->model, in5, Min, h->ncell, h->d_pad_cell, h->d_pad_src, h->npad, h->stream);
        } else {
            launch_fill_pads(h->D, h->model, h->p.inlet, Min, h->ncell, h->d_pad_cell, h->d_pad_src, h->npad,
                             h->stream);
        }
        CUDA_TRY(h, cudaMemsetAsync(Mout, 0, bytes, h->stream));
        CUDA_TRY(h, cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), h->stream));
        std::pair<cudaEvent_t, cudaEvent_t> ev{};
        if (h->timing) {
            int rc = take_events(h, &ev);
            if (rc) return rc;
            CUDA_TRY(h, cudaEventRecord(ev.first, h->stream));
        }
        // the learned warm start runs as its own kernel; the cell update reads its output
        // (timed with the cell update: it is part of the learned start's cost)
        Model mc = h->model;
        if (mc.mlp_w) {
            launch_mlp_start(mc, h->geo, h->d_type, Min, h->d_mlp_start, h->device, h->stream);
            mc.mlp_start = h->d_mlp_start;
            mc.mlp_w = nullptr;
            mc.mlp_nrm = nullptr;
        }
        if (h->d_det_lam) {
            mc.det_lam = h->d_det_lam;
            mc.det_halo = h->d_det_halo;
            CUDA_TRY(h, cudaMemsetAsync(h->d_det_halo, 0, sizeof(int), h->stream));
        }
        if (h->D == 3)
            launch_cell3d(mc, h->geo3, Min, Mout, h->d_stats, h->d_work, h->blocks, h->stream);
        else
            launch_cell_update(mc, h->geo, h->d_type, Min, Mout, h->d_stats, h->d_work, h->blocks, h->p.precision,
                               h->stream);
        if (h->d_det_lam) launch_gather2d(mc, h->geo, Min, Mout, h->d_stats, h->stream);
        if (h->timing) {
            CUDA_TRY(h, cudaEventRecord(ev.second, h->stream));
            h->ev_used.push_back(ev);
        }
        CUDA_TRY(h, cudaGetLastError());
        h->cur = 1 - h->cur;
        h->steps++;
    }
    return LELBM_OK;
}

static int read_stats(lelbm* h, lelbm_stats* s) {
    DevStats d;
    CUDA_TRY(h, cudaMemcpyAsync(&d, h->d_stats, sizeof d, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    int rc = collect_timing(h);
    if (rc) return rc;
    if (s) {
        std::memset(s, 0, sizeof *s);
        s->steps = h->steps;
        s->cells = (long long)d.cells;
        for (int i = 0; i < 64; i++) s->newton_hist[i] = (long long)d.newton_hist[i];
        s->fallback_eq = (long long)d.fallback_eq;
        s->fallback_mx = (long long)d.fallback_mx;
        s->q_max = (long long)d.q_max;
        double dm;
        std::memcpy(&dm, &d.disp_max_bits, sizeof dm);
        s->disp_max = dm;
        s->first_fail_cell = d.first_fail == ~0ull ? -1 : (long long)d.first_fail;
        s->cell_kernel_ms = h->timed_ms;
        s->cell_kernel_launches = h->timed_launches;
        s->points_f = (long long)d.points_f;
        s->points_g = (long long)d.points_g;
        s->points_ms = (long long)d.points_ms;
        s->points_32 = (long long)d.points_32;
        s->judge_redo = (long long)d.judge_redo;
        s->mlp_retry = (long long)d.mlp_retry;
        s->wall_hits = (long long)d.wall_hits;
        s->mlp_cells = (long long)d.mlp_cells;
        s->points_df = (long long)d.points_df;
        s->points_df_corr = (long long)d.points_df_corr;
    }
    return d.fallback_mx ? LELBM_E_EPR : LELBM_OK;
}

extern "C" int lelbm_synchronize(lelbm_t h) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    int rc = read_stats(h, nullptr);
    if (rc == LELBM_E_EPR) return fail(h, LELBM_E_EPR, "EPR fell back to Maxwellian weights");
    return rc;
}

extern "C" int lelbm_get_moments(lelbm_t h, double* m) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!m) return fail(h, LELBM_E_INVAL, "NULL output");
    const size_t bytes = sizeof(double) * (size_t)h->nmom * (size_t)h->ncell;
    CUDA_TRY(h, cudaMemcpyAsync(m, h->M[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LELBM_OK;
}

extern "C" int lelbm_get_moments_device(lelbm_t h, double* m_dev) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!m_dev) return fail(h, LELBM_E_INVAL, "NULL output");
    const size_t bytes = sizeof(double) * (size_t)h->nmom * (size_t)h->ncell;
    CUDA_TRY(h, cudaMemcpyAsync(m_dev, h->M[h->cur], bytes, cudaMemcpyDeviceToDevice, h->stream));
    return LELBM_OK;
}

extern "C" int lelbm_get_macros(lelbm_t h, double* rho, double* u, double* RT) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!rho || !u || !RT) return fail(h, LELBM_E_INVAL, "NULL output");
    const long long n = h->ncell;
    double* d = nullptr;
    CUDA_TRY(h, cudaMalloc((void**)&d, sizeof(double) * n * (2 + h->D)));
    launch_macros(h->D, h->model.K, h->d_type, h->M[h->cur], d, d + n, d + n * (1 + h->D), n, h->stream);
    cudaMemcpyAsync(rho, d, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(u, d + n, sizeof(double) * n * h->D, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(RT, d + n * (1 + h->D), sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(h, LELBM_E_CUDA, "get_macros: %s", cudaGetErrorString(e));
    return LELBM_OK;
}

extern "C" int lelbm_get_stats(lelbm_t h, lelbm_stats* s) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!s) return fail(h, LELBM_E_INVAL, "NULL output");
    int rc = read_stats(h, s);
    return rc == LELBM_E_EPR ? LELBM_OK : rc;
}

extern "C" int lelbm_reset_stats(lelbm_t h) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    int rc = collect_timing(h);
    if (rc) return rc;
    return reset_stats_dev(h);
}

extern "C" int lelbm_set_timing(lelbm_t h, int on) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    h->timing = on != 0;
    return LELBM_OK;
}

extern "C" int lelbm_set_steps(lelbm_t h, const int* steps) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (h->D != 1) return fail(h, LELBM_E_INVAL, "step budgets are for 1D batches");
    const int nb = (int)h->inst_n_h.size();
    if (!steps) {
        h->budgets = false;
        return LELBM_OK;
    }
    for (int b = 0; b < nb; b++)
        if (steps[b] < 0) return fail(h, LELBM_E_INVAL, "steps[%d] < 0", b);
    if (!h->d_steps_left) CUDA_TRY(h, cudaMalloc((void**)&h->d_steps_left, sizeof(int) * nb));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_steps_left, steps, sizeof(int) * nb, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->budgets = true;
    return LELBM_OK;
}

static int tuned_blocks(lelbm* h, const lelbm_tuning& t) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const int mx = batch_persistent_max_blocks_per_sm(h->p.precision, t.threads);
    const int per = (t.blocks_per_sm <= 0 || t.blocks_per_sm > mx) ? mx : t.blocks_per_sm;
    return sms * per;
}

// Enqueue one persistent launch (work-counter reset + kernel) on the handle's stream.
static int enqueue_batch(lelbm* h, int n, const lelbm_tuning& t) {
    CUDA_TRY(h, cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), h->stream));
    launch_batch_persistent(h->model, h->geo, h->p.inlet, h->p.bc[0] == LELBM_BC_INFLOW,
                            h->p.bc[1] == LELBM_BC_INFLOW, h->d_type, h->M[h->cur], h->M[1 - h->cur], h->d_stats,
                            h->d_work, h->d_order[t.order ? 1 : 0], h->d_inst_first, h->d_inst_pad,
                            h->budgets ? h->d_steps_left : nullptr, n, tuned_blocks(h, t), t.threads,
                            h->p.precision, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    return LELBM_OK;
}

extern "C" int lelbm_run_batch(lelbm_t h, int n) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (h->D != 1) return fail(h, LELBM_E_INVAL, "lelbm_run_batch needs a 1D handle");
    if (n < 0) return fail(h, LELBM_E_INVAL, "n must be >= 0");
    if (n == 0) return LELBM_OK;
    const lelbm_tuning& t = h->tuning;
    // the graph holds the buffer pointers, the launch shape, n and the budget pointer
    const bool same = h->graph && h->graph_n == n && h->graph_cur == h->cur && h->graph_budgets == h->budgets &&
                      h->graph_tuning.threads == t.threads && h->graph_tuning.blocks_per_sm == t.blocks_per_sm &&
                      h->graph_tuning.order == t.order;
    if (!same) {
        if (h->graph) cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        cudaGraph_t gr = nullptr;
        CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_batch(h, n, t);
        cudaError_t e = cudaStreamEndCapture(h->stream, &gr);
        if (rc) return rc;
        if (e != cudaSuccess) return fail(h, LELBM_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->graph, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return fail(h, LELBM_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        h->graph_n = n;
        h->graph_cur = h->cur;
        h->graph_budgets = h->budgets;
        h->graph_tuning = t;
    }
    std::pair<cudaEvent_t, cudaEvent_t> ev{};
    if (h->timing) {
        int rc = take_events(h, &ev);
        if (rc) return rc;
        CUDA_TRY(h, cudaEventRecord(ev.first, h->stream));
    }
    CUDA_TRY(h, cudaGraphLaunch(h->graph, h->stream));
    if (h->timing) {
        CUDA_TRY(h, cudaEventRecord(ev.second, h->stream));
        h->ev_used.push_back(ev);
    }
    h->steps += n;
    return LELBM_OK;
}

extern "C" int lelbm_set_tuning(lelbm_t h, const lelbm_tuning* t) {
    if (!h || !t) return fail(h, LELBM_E_INVAL, "NULL argument");
    if ((t->threads != 64 && t->threads != 128) || t->blocks_per_sm < 0 || (t->order != 0 && t->order != 1))
        return fail(h, LELBM_E_INVAL, "bad tuning");
    h->tuning = *t;
    h->tuning.ms = 0.0;
    return LELBM_OK;
}

extern "C" int lelbm_autotune(lelbm_t h, int trial_steps, lelbm_tuning* best) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (h->D != 1) return fail(h, LELBM_E_INVAL, "lelbm_autotune needs a 1D handle");
    if (trial_steps < 1) return fail(h, LELBM_E_INVAL, "trial_steps must be >= 1");
    const size_t bytes = sizeof(double) * (size_t)h->nmom * (size_t)h->ncell;
    const int nb = (int)h->inst_n_h.size();
    double* save = nullptr;
    int* save_steps = nullptr;
    float* save_lam = nullptr;  // the stored warm start is state the trials change too
    const size_t lam_bytes = sizeof(float) * 7 * (size_t)h->ncell;
    CUDA_TRY(h, cudaMalloc((void**)&save, bytes));
    if ((h->budgets && cudaMalloc((void**)&save_steps, sizeof(int) * nb) != cudaSuccess) ||
        (h->d_lam && cudaMalloc((void**)&save_lam, lam_bytes) != cudaSuccess)) {
        cudaFree(save);
        cudaFree(save_steps);
        return fail(h, LELBM_E_NOMEM, "autotune backup");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int mx128 = batch_persistent_max_blocks_per_sm(h->p.precision, 128);
    std::vector<lelbm_tuning> cand;
    for (int threads : {64, 128})
        for (int per : {1, 2, 0})
            for (int order : {0, 1}) {
                if (threads == 128 && per == 2 && mx128 < 2) continue;
                cand.push_back({threads, per, order, 0.0});
            }
    lelbm_tuning win{128, 0, 0, 1e300};
    int rc = LELBM_OK;
    cudaMemcpyAsync(save, h->M[h->cur], bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (save_steps) cudaMemcpyAsync(save_steps, h->d_steps_left, sizeof(int) * nb, cudaMemcpyDeviceToDevice, h->stream);
    if (save_lam) cudaMemcpyAsync(save_lam, h->d_lam, lam_bytes, cudaMemcpyDeviceToDevice, h->stream);
    for (auto& t : cand) {
        cudaEventRecord(e0, h->stream);
        rc = enqueue_batch(h, trial_steps, t);
        if (rc) break;
        cudaEventRecord(e1, h->stream);
        cudaMemcpyAsync(h->M[h->cur], save, bytes, cudaMemcpyDeviceToDevice, h->stream);
        if (save_steps)
            cudaMemcpyAsync(h->d_steps_left, save_steps, sizeof(int) * nb, cudaMemcpyDeviceToDevice, h->stream);
        if (save_lam) cudaMemcpyAsync(h->d_lam, save_lam, lam_bytes, cudaMemcpyDeviceToDevice, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = fail(h, LELBM_E_CUDA, "autotune trial failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t.ms = ms;
        if (ms < win.ms) win = t;
    }
    cudaStreamSynchronize(h->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(save);
    cudaFree(save_steps);
    cudaFree(save_lam);
    if (rc) return rc;
    h->tuning = win;
    int r2 = reset_stats_dev(h);
    if (r2) return r2;
    if (best) *best = win;
    return LELBM_OK;
}

extern "C" int lelbm_step_record(lelbm_t h, float* x_dev, float* y_dev) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!x_dev || !y_dev) return fail(h, LELBM_E_INVAL, "NULL record buffer");
    if (h->D == 3) return fail(h, LELBM_E_INVAL, "training pairs are recorded in 1D and 2D");
    h->model.rec_x = x_dev;
    h->model.rec_y = y_dev;
    const int rc = lelbm_step(h, 1);
    h->model.rec_x = nullptr;
    h->model.rec_y = nullptr;
    return rc;
}

extern "C" int lelbm_set_warmstart(lelbm_t h, int stored) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (h->D == 3 && stored) return fail(h, LELBM_E_INVAL, "3D has no warm-start store");
    if (stored) {
        if (!h->d_lam) {
            const size_t bytes = sizeof(float) * (size_t)(h->D == 1 ? 7 : 16) * (size_t)h->ncell;
            CUDA_TRY(h, cudaMalloc((void**)&h->d_lam, bytes));
            CUDA_TRY(h, cudaMemsetAsync(h->d_lam, 0, bytes, h->stream));
            CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        }
        h->model.lam_store = h->d_lam;
    } else {
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->d_lam);
        h->d_lam = nullptr;
        h->model.lam_store = nullptr;
    }
    if (h->graph) cudaGraphExecDestroy(h->graph);  // the captured launch holds the old model
    h->graph = nullptr;
    return LELBM_OK;
}

extern "C" int lelbm_set_mlp_gate(lelbm_t h, double departure) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    if (!(departure >= 0.0) || !std::isfinite(departure)) return fail(h, LELBM_E_INVAL, "departure must be >= 0");
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->model.mlp_gate = (float)departure;
    if (h->graph) cudaGraphExecDestroy(h->graph);  // the captured launch holds the old model
    h->graph = nullptr;
    return LELBM_OK;
}

extern "C" int lelbm_set_mlp(lelbm_t h, const float* params) {
    if (!h) return fail(nullptr, LELBM_E_INVAL, "handle is NULL");
    int nin, nout;
    long long ntot, nw;
    if (lelbm_mlp_size(h->D, &nin, &nout, &ntot, &nw) != LELBM_OK) return fail(h, LELBM_E_INVAL, "bad dims");
    if (!params) {
        h->model.mlp_w = nullptr;
        h->model.mlp_nrm = nullptr;
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->d_mlp_start);
        h->d_mlp_start = nullptr;
        if (h->graph) cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        return LELBM_OK;
    }
    for (long long i = 0; i < ntot; i++)
        if (!std::isfinite(params[i])) return fail(h, LELBM_E_INVAL, "non-finite MLP parameter %lld", i);
    std::vector<__nv_bfloat16> w(nw);
    for (long long i = 0; i < nw; i++) w[i] = __float2bfloat16(params[i]);
    if (!h->d_mlp_w) CUDA_TRY(h, cudaMalloc((void**)&h->d_mlp_w, sizeof(__nv_bfloat16) * nw));
    if (!h->d_mlp_nrm) CUDA_TRY(h, cudaMalloc((void**)&h->d_mlp_nrm, sizeof(float) * (ntot - nw)));
    if (!h->d_mlp_start) CUDA_TRY(h, cudaMalloc((void**)&h->d_mlp_start, sizeof(float) * (size_t)nout * h->ncell));
    CUDA_TRY(h, cudaMemcpy(h->d_mlp_w, w.data(), sizeof(__nv_bfloat16) * nw, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->d_mlp_nrm, params + nw, sizeof(float) * (ntot - nw), cudaMemcpyHostToDevice));
    h->model.mlp_w = h->d_mlp_w;
    h->model.mlp_nrm = h->d_mlp_nrm;
    if (h->graph) cudaGraphExecDestroy(h->graph);  // the captured launch holds the old model
    h->graph = nullptr;
    return LELBM_OK;
}

extern "C" const char* lelbm_last_error(lelbm_t h) { return h ? h->err.c_str() : g_create_err.c_str(); }

extern "C" int lelbm_fma_peak(int fp64, double* flops) {
    if (!flops) return fail(nullptr, LELBM_E_INVAL, "flops is NULL");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, LELBM_E_CUDA, "no CUDA device");
    const double v = fma_peak(fp64, dev);
    if (v < 0.0) return fail(nullptr, LELBM_E_CUDA, "FMA probe failed");
    *flops = v;
    return LELBM_OK;
}

extern "C" int lelbm_mlp_infer(int dims, const float* params, const float* X_dev, long long n, float* Y_dev,
                               void* stream) {
    int nin, nout;
    long long ntot, nw;
    if (lelbm_mlp_size(dims, &nin, &nout, &ntot, &nw) != LELBM_OK) return fail(nullptr, LELBM_E_INVAL, "bad dims");
    if (!params || n < 0 || (n > 0 && (!X_dev || !Y_dev))) return fail(nullptr, LELBM_E_INVAL, "bad argument");
    if (n == 0) return LELBM_OK;
    std::vector<__nv_bfloat16> w(nw);
    for (long long i = 0; i < nw; i++) w[i] = __float2bfloat16(params[i]);
    __nv_bfloat16* dw = nullptr;
    float* dn = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMalloc((void**)&dw, sizeof(__nv_bfloat16) * nw) != cudaSuccess ||
        cudaMalloc((void**)&dn, sizeof(float) * (ntot - nw)) != cudaSuccess) {
        cudaFree(dw);
        return fail(nullptr, LELBM_E_NOMEM, "device allocation failed");
    }
    cudaMemcpyAsync(dw, w.data(), sizeof(__nv_bfloat16) * nw, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dn, params + nw, sizeof(float) * (ntot - nw), cudaMemcpyHostToDevice, s);
    launch_mlp_infer(dims, dw, dn, X_dev, n, Y_dev, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(dw);
    cudaFree(dn);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(nullptr, LELBM_E_CUDA, "MLP inference failed");
    return LELBM_OK;
}
