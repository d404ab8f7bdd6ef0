// C ABI of liboreg.so (declared in include/oreg.h): lattice objects, parameter
// validation, memory ownership, error reporting and dispatch to the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "oreg.h"
#include "oreg_consts.h"
#include "oreg_device.cuh"
#include "oreg_launch.h"
#include "oreg_lattice.h"

using namespace oreg;

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
namespace {
thread_local std::string g_last_error;

olb_status fail(olb_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

olb_status cuda_fail(cudaError_t e, const char *what) {
    // a failed allocation is not sticky, but it stays the thread's last error:
    // clear it, so that the next launch check of this thread does not report it
    if (e == cudaErrorMemoryAllocation) (void)cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? OLB_ERR_NOMEM : OLB_ERR_CUDA, "%s: %s (%s)",
                what, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define OLB_CUDA(call, what)                                 \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);   \
    } while (0)

size_t elem_size(int storage) {
    switch (storage) {
        case OLB_F64: return 8;
        case OLB_F32: return 4;
        case OLB_F16_SHIFTED:
        case OLB_BF16_SHIFTED: return 2;
        default: return 0;
    }
}

int vec_elems(int storage) { return 16 / (int)elem_size(storage); }

constexpr size_t CHUNK_BYTES_MAX = size_t(64) << 20;  // readback scratch
}  // namespace

namespace oreg {
// Records the message of a failed call made outside this file (the
// no-allocation diagnostics entry point) for olb_last_error().
void set_last_error_message(const char *msg) { g_last_error = msg; }
}  // namespace oreg


namespace {

olb_status validate(const olb_params *p) {
    if (!p) return fail(OLB_ERR_INVALID, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(OLB_ERR_INVALID, "nx, ny must be >= 1 (got %d, %d)", p->nx, p->ny);
    if ((int64_t)p->nx * p->ny > (int64_t)1 << 36)
        return fail(OLB_ERR_INVALID, "lattice too large: %d x %d", p->nx, p->ny);
    if (!(std::isfinite(p->tau) && p->tau > 0.5))
        return fail(OLB_ERR_INVALID, "tau must be finite and > 0.5 (got %g)", p->tau);
    if (!(std::isfinite(p->rho0) && p->rho0 > 0))
        return fail(OLB_ERR_INVALID, "rho0 must be finite and > 0 (got %g)", p->rho0);
    if (p->eq != OLB_EQ_GUIDED && p->eq != OLB_EQ_POLY2)
        return fail(OLB_ERR_INVALID, "unknown equilibrium %d", p->eq);
    if (p->coll != OLB_COLL_OREG && p->coll != OLB_COLL_BGK)
        return fail(OLB_ERR_INVALID, "unknown collision %d", p->coll);
    if (elem_size(p->storage) == 0) return fail(OLB_ERR_INVALID, "unknown storage %d", p->storage);
    {
        // the kernels index the 16-byte vectors of a population plane with an int
        const int V = vec_elems(p->storage);
        if ((int64_t)((p->nx + V - 1) / V) * p->ny > (int64_t)INT32_MAX - 64)
            return fail(OLB_ERR_INVALID, "lattice too large: %d x %d (over 2^31 vectors per plane)",
                        p->nx, p->ny);
    }
    if (p->layout != OLB_LAYOUT_AB && p->layout != OLB_LAYOUT_AA)
        return fail(OLB_ERR_INVALID, "unknown layout %d", p->layout);
    if (p->eq == OLB_EQ_GUIDED && !(p->theta > 0 && p->theta < 1))
        return fail(OLB_ERR_INVALID, "guided equilibrium needs 0 < theta < 1 (got %g)", p->theta);
    if (p->eq == OLB_EQ_POLY2 && std::fabs(p->theta - 1.0 / 3.0) > 1e-12)
        return fail(OLB_ERR_INVALID, "polynomial equilibrium is defined at theta = 1/3 only (got %.17g)", p->theta);
    if (p->boundary != OLB_BOUNDARY_PERIODIC && p->boundary != OLB_BOUNDARY_WALLS_X)
        return fail(OLB_ERR_INVALID, "unknown boundary %d", p->boundary);
    if (p->boundary == OLB_BOUNDARY_WALLS_X && p->nx < 3)
        return fail(OLB_ERR_INVALID, "wall columns need nx >= 3 (got %d)", p->nx);
    if (p->theta_mode != OLB_THETA_FIXED && p->theta_mode != OLB_THETA_LOCAL)
        return fail(OLB_ERR_INVALID, "unknown theta mode %d", p->theta_mode);
    if (p->theta_mode == OLB_THETA_LOCAL && p->eq != OLB_EQ_GUIDED)
        return fail(OLB_ERR_INVALID, "the local temperature needs the guided equilibrium");
    return OLB_OK;
}

int pitch_of(const olb_params *p) {
    const int V = vec_elems(p->storage);
    return ((p->nx + V - 1) / V) * V;
}

size_t pop_bytes(const olb_params *p) {
    const size_t plane = (size_t)pitch_of(p) * p->ny;
    const int nbuf = p->layout == OLB_LAYOUT_AB ? 2 : 1;
    return (size_t)nbuf * 9 * plane * elem_size(p->storage);
}

#define DISPATCH(storage, fn, ...)                                      \
    ((storage) == OLB_F64   ? fn##_f64(__VA_ARGS__)                     \
     : (storage) == OLB_F32 ? fn##_f32(__VA_ARGS__)                     \
     : (storage) == OLB_F16_SHIFTED ? fn##_f16(__VA_ARGS__)             \
                                    : fn##_bf16(__VA_ARGS__))

olb_status check_lattice(const olb_lattice *L, bool need_state) {
    if (!L) return fail(OLB_ERR_INVALID, "lattice is NULL");
    if (L->batch && !need_state)
        return fail(OLB_ERR_STATE, "lattice belongs to a batch: remove it before re-initialising");
    if (need_state && L->t < 0) return fail(OLB_ERR_STATE, "lattice state not initialised (call an olb_init_* first)");
    return OLB_OK;
}

olb_status ensure_chunk(olb_lattice *L, size_t bytes) {
    if (L->chunk_bytes >= bytes) return OLB_OK;
    if (L->d_chunk) {
        cudaStreamSynchronize(L->stream);
        if (L->copy_stream) cudaStreamSynchronize(L->copy_stream);
        cudaFree(L->d_chunk);
        L->d_chunk = nullptr;
        L->chunk_bytes = 0;
    }
    OLB_CUDA(cudaMalloc(&L->d_chunk, bytes), "allocating readback scratch");
    L->chunk_bytes = bytes;
    return OLB_OK;
}

// Staged transfers queue their copies asynchronously and wait once at the
// end; this guard also waits when a call returns early on an error, so that no
// queued copy still reads or writes the caller's host arrays after the return.
struct StreamDrain {
    cudaStream_t s;
    ~StreamDrain() {
        if (s) cudaStreamSynchronize(s);
    }
};

// The copy stream and events of the double-buffered field upload and moments
// readback (created on first use, released by olb_destroy).
olb_status ensure_pipeline(olb_lattice *L) {
    if (L->copy_stream) return OLB_OK;
    OLB_CUDA(cudaStreamCreateWithFlags(&L->copy_stream, cudaStreamNonBlocking), "creating copy stream");
    for (int b = 0; b < 2; ++b) {
        OLB_CUDA(cudaEventCreateWithFlags(&L->ev_main[b], cudaEventDisableTiming), "creating event");
        OLB_CUDA(cudaEventCreateWithFlags(&L->ev_copy[b], cudaEventDisableTiming), "creating event");
    }
    return OLB_OK;
}

// rows per readback chunk for `per_node_doubles` FP64 values per node
int chunk_rows(const olb_lattice *L, int per_node_doubles) {
    const size_t row_bytes = (size_t)L->p.nx * per_node_doubles * sizeof(double);
    size_t rows = CHUNK_BYTES_MAX / row_bytes;
    if (rows < 1) rows = 1;
    if (rows > (size_t)L->p.ny) rows = L->p.ny;
    return (int)rows;
}

olb_status run_init(olb_lattice *L, InitSpec spec) {
    L->t = 0;
    const StateGeom g = geom(L);
    void *base = state_base(L);
    if (spec.mode != INIT_FIELDS) {
        spec.y0 = 0;
        spec.rows = L->p.ny;
    }
    OLB_CUDA(DISPATCH(L->p.storage, init, base, g, spec, L->p.eq, L->kd, L->stream),
             "launching init kernel");
    return OLB_OK;
}

// Reduction partials and the pinned result buffer, allocated on first use (a
// lattice whose owner never asks for a reduction never allocates them).
olb_status ensure_reduction(olb_lattice *L) {
    if (L->d_red) return OLB_OK;
    OLB_CUDA(cudaMalloc(&L->d_red, ((size_t)RED_BLOCKS_MAX + 1) * RED_QUANTITIES * sizeof(double)),
             "allocating reduction scratch");
    cudaError_t e = cudaMallocHost(&L->h_red, RED_QUANTITIES * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(L->d_red);
        L->d_red = nullptr;
        L->h_red = nullptr;
        return cuda_fail(e, "allocating pinned result buffer");
    }
    return OLB_OK;
}

olb_status reduce(olb_lattice *L, const ModeSpec &mode, double out[RED_QUANTITIES]) {
    olb_status st = ensure_reduction(L);
    if (st != OLB_OK) return st;
    const StateGeom g = geom(L);
    double *partials = L->d_red;
    double *dres = L->d_red + (size_t)RED_BLOCKS_MAX * RED_QUANTITIES;
    OLB_CUDA(DISPATCH(L->p.storage, reduce, state_base(L), g, L->kd, mode, partials,
                      L->red_blocks, dres, L->stream),
             "launching reduction");
    OLB_CUDA(cudaMemcpyAsync(L->h_red, dres, RED_QUANTITIES * sizeof(double),
                             cudaMemcpyDeviceToHost, L->stream),
             "copying reduction result");
    OLB_CUDA(cudaStreamSynchronize(L->stream), "synchronising reduction");
    for (int q = 0; q < RED_QUANTITIES; ++q) out[q] = L->h_red[q];
    // the kernel sums the shifted values g; add the shifts of the finite nodes
    double sum_shift = 0.0;
    for (int i = 0; i < 9; ++i) sum_shift += L->kd.shift[dcls(i)];
    const double n_finite = (double)L->p.nx * L->p.ny - out[3];
    out[0] += n_finite * sum_shift;
    return OLB_OK;
}

// FP64 tables sin/cos(2 pi m x / nx) and sin/cos(2 pi n y / ny) for the
// mode projection, rebuilt when (m, n) changes.
olb_status mode_tables(olb_lattice *L, int m, int n) {
    const size_t cnt = 2 * ((size_t)L->p.nx + L->p.ny);
    if (!L->d_tab) {
        OLB_CUDA(cudaMalloc(&L->d_tab, cnt * sizeof(double)), "allocating mode tables");
        OLB_CUDA(cudaMallocHost(&L->h_tab, cnt * sizeof(double)), "allocating mode tables");
        L->tab_m = L->tab_n = 0;
    } else if (L->tab_m == m && L->tab_n == n) {
        return OLB_OK;
    }
    const int nx = L->p.nx, ny = L->p.ny;
    const double two_pi = 6.283185307179586476925286766559;
    for (int x = 0; x < nx; ++x) {
        const long long r = ((long long)m * x) % nx;
        const double a = two_pi * (double)(r < 0 ? r + nx : r) / nx;
        L->h_tab[x] = std::sin(a);
        L->h_tab[nx + x] = std::cos(a);
    }
    for (int y = 0; y < ny; ++y) {
        const long long r = ((long long)n * y) % ny;
        const double b = two_pi * (double)(r < 0 ? r + ny : r) / ny;
        L->h_tab[2 * nx + y] = std::sin(b);
        L->h_tab[2 * nx + ny + y] = std::cos(b);
    }
    OLB_CUDA(cudaMemcpyAsync(L->d_tab, L->h_tab, cnt * sizeof(double), cudaMemcpyHostToDevice,
                             L->stream),
             "copying mode tables");
    L->tab_m = m;
    L->tab_n = n;
    return OLB_OK;
}

}  // namespace

extern "C" {

int32_t olb_abi_version(void) { return 5; }

size_t olb_required_bytes(const olb_params *p) {
    if (validate(p) != OLB_OK) return 0;
    return pop_bytes(p);
}

olb_status olb_create_lattice(const olb_params *p, olb_lattice **out) {
    if (!out) return fail(OLB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    olb_status st = validate(p);
    if (st != OLB_OK) return st;
    const size_t need = pop_bytes(p);
    if (p->device_buffer) {
        if (p->buffer_bytes < need)
            return fail(OLB_ERR_INVALID, "device_buffer holds %zu bytes, %zu needed", p->buffer_bytes, need);
        if (reinterpret_cast<uintptr_t>(p->device_buffer) % 256 != 0)
            return fail(OLB_ERR_INVALID, "device_buffer must be 256-byte aligned");
    }
    olb_lattice *L = new (std::nothrow) olb_lattice();
    if (!L) return fail(OLB_ERR_NOMEM, "host allocation of the lattice failed");
    L->p = *p;
    L->esize = elem_size(p->storage);
    L->V = vec_elems(p->storage);
    L->pitch = pitch_of(p);
    L->plane = (size_t)L->pitch * p->ny;
    L->buf_elems = 9 * L->plane;
    L->nbuf = p->layout == OLB_LAYOUT_AB ? 2 : 1;
    L->t = -1;
    L->comp = p->storage == OLB_F32 ? 1 : 0;
    L->f64_coll = 0;
    L->sr = (p->storage == OLB_F16_SHIFTED || p->storage == OLB_BF16_SHIFTED) ? 1 : 0;
    L->warps_per_block = 4;
    L->kd = make_const_f64_for(p);
    L->kf = make_step_const_f32(p);

    auto bail = [&](olb_status s) {
        olb_destroy(L);
        return s;
    };
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&L->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bail(cuda_fail(e, "querying the device"));
    if (p->cuda_stream) {
        L->stream = static_cast<cudaStream_t>(p->cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&L->owned_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(e, "creating the stream"));
        L->stream = L->owned_stream;
    }
    if (p->device_buffer) {
        L->mem = p->device_buffer;
        L->own_mem = false;
    } else {
        e = cudaMalloc(&L->mem, need);
        if (e != cudaSuccess) {
            L->mem = nullptr;
            return bail(cuda_fail(e, "allocating population memory"));
        }
        L->own_mem = true;
    }
    // zero the populations (keeps row padding finite); stream-ordered
    e = cudaMemsetAsync(L->mem, 0, need, L->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "clearing population memory"));
    const long long N = (long long)p->nx * p->ny;
    long long blocks = (N + 255) / 256;
    const long long cap = std::min<long long>(RED_BLOCKS_MAX, 8LL * L->num_sms);
    L->red_blocks = (int)std::max<long long>(1, std::min(blocks, cap));
    // the reduction scratch is allocated by the first reduction (ensure_reduction)
    *out = L;
    return OLB_OK;
}

olb_status olb_set_stream(olb_lattice *L, void *cuda_stream) {
    if (!L) return fail(OLB_ERR_INVALID, "lattice is NULL");
    if (L->batch)
        return fail(OLB_ERR_STATE, "a batch member runs on the batch's stream: remove it first");
    if (cuda_stream) {
        L->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (!L->owned_stream)
            return fail(OLB_ERR_INVALID, "the lattice was created on a caller stream: pass a stream");
        L->stream = L->owned_stream;
    }
    return OLB_OK;
}

olb_status olb_set_option(olb_lattice *L, int32_t option, int64_t value) {
    olb_status st = check_lattice(L, false);
    if (st != OLB_OK) return st;
    switch (option) {
        case OLB_OPT_COMPENSATED:
            if (value != 0 && value != 1) return fail(OLB_ERR_INVALID, "OLB_OPT_COMPENSATED takes 0 or 1");
            L->comp = (int)value;
            return OLB_OK;
        case OLB_OPT_STOCHASTIC_ROUNDING:
            if (value != 0 && value != 1) return fail(OLB_ERR_INVALID, "OLB_OPT_STOCHASTIC_ROUNDING takes 0 or 1");
            L->sr = (int)value;
            return OLB_OK;
        case OLB_OPT_F64_COLLISION:
            if (value != 0 && value != 1) return fail(OLB_ERR_INVALID, "OLB_OPT_F64_COLLISION takes 0 or 1");
            if (value == 1 && L->p.storage != OLB_F32)
                return fail(OLB_ERR_INVALID, "OLB_OPT_F64_COLLISION needs OLB_F32 storage");
            L->f64_coll = (int)value;
            return OLB_OK;
        case OLB_OPT_WARPS_PER_BLOCK:
            if (value < 1 || value > 8 || (value & (value - 1)))
                return fail(OLB_ERR_INVALID, "OLB_OPT_WARPS_PER_BLOCK takes 1, 2, 4 or 8");
            L->warps_per_block = (int)value;
            return OLB_OK;
        default: return fail(OLB_ERR_INVALID, "unknown option %d", option);
    }
}

olb_status olb_init_shear_flow(olb_lattice *L, double rho0, double u0, int32_t m, int32_t n,
                               double ux_mean, double uy_mean, int32_t first_order) {
    olb_status st = check_lattice(L, false);
    if (st != OLB_OK) return st;
    if (m == 0 && n == 0) return fail(OLB_ERR_INVALID, "wave vector (m, n) must not be (0, 0)");
    if (!(std::isfinite(rho0) && rho0 > 0 && std::isfinite(u0)))
        return fail(OLB_ERR_INVALID, "rho0 must be > 0 and u0 finite");
    if (!(std::isfinite(ux_mean) && std::isfinite(uy_mean)))
        return fail(OLB_ERR_INVALID, "mean flow must be finite");
    if (first_order != 0 && first_order != 1)
        return fail(OLB_ERR_INVALID, "first_order must be 0 or 1 (got %d)", first_order);
    InitSpec s{};
    s.mode = INIT_SHEAR;
    s.rho_a = rho0;
    s.u0 = u0;
    s.m = m;
    s.n = n;
    const double kx = (double)m / L->p.nx, ky = (double)n / L->p.ny;
    const double nk = std::hypot(kx, ky);
    s.ex = -ky / nk;
    s.ey = kx / nk;
    s.ux_mean = ux_mean;
    s.uy_mean = uy_mean;
    s.first_order = first_order;
    const double two_pi = 6.283185307179586476925286766559;
    s.kx = two_pi * kx;
    s.ky = two_pi * ky;
    s.tau = L->p.tau;
    return run_init(L, s);
}

olb_status olb_init_shear_wave(olb_lattice *L, double rho0, double u0, int32_t m, int32_t n) {
    return olb_init_shear_flow(L, rho0, u0, m, n, 0.0, 0.0, 0);
}

olb_status olb_init_shock_tube(olb_lattice *L, double rho_left, double rho_right, int32_t x_split) {
    olb_status st = check_lattice(L, false);
    if (st != OLB_OK) return st;
    if (!(rho_left > 0 && rho_right > 0 && std::isfinite(rho_left) && std::isfinite(rho_right)))
        return fail(OLB_ERR_INVALID, "densities must be finite and > 0");
    InitSpec s{};
    s.mode = INIT_SHOCK;
    s.rho_a = rho_left;
    s.rho_b = rho_right;
    s.x_split = x_split;
    return run_init(L, s);
}

olb_status olb_init_fields(olb_lattice *L, const double *rho, const double *ux, const double *uy) {
    oreg::NvtxRange nvtx_("olb_init_fields");
    olb_status st = check_lattice(L, false);
    if (st != OLB_OK) return st;
    if (!rho || !ux || !uy) return fail(OLB_ERR_INVALID, "field arrays must not be NULL");
    // fields are staged through the bounded readback scratch, a chunk of rows
    // at a time, alternating between its two halves: the copies of chunk k
    // (copy stream) overlap the conversion kernel of chunk k-1 (lattice stream)
    const int rows = chunk_rows(L, 3);
    const size_t nx = L->p.nx, half = (size_t)rows * nx * 3;
    st = ensure_chunk(L, 2 * half * sizeof(double));
    if (st != OLB_OK) return st;
    st = ensure_pipeline(L);
    if (st != OLB_OK) return st;
    double *base = static_cast<double *>(L->d_chunk);
    StreamDrain drain_{L->stream}, drain_copy_{L->copy_stream};
    // copies into either half wait for the lattice stream's earlier work
    for (int b = 0; b < 2; ++b)
        OLB_CUDA(cudaEventRecord(L->ev_main[b], L->stream), "recording event");
    for (int y0 = 0, k = 0; y0 < L->p.ny; y0 += rows, ++k) {
        const int b = k & 1;
        double *d = base + b * half;
        const int r = std::min(rows, L->p.ny - y0);
        const size_t cnt = (size_t)r * nx, off = (size_t)y0 * nx;
        OLB_CUDA(cudaStreamWaitEvent(L->copy_stream, L->ev_main[b], 0), "ordering copy");
        OLB_CUDA(cudaMemcpyAsync(d, rho + off, cnt * sizeof(double), cudaMemcpyHostToDevice, L->copy_stream), "copying rho");
        OLB_CUDA(cudaMemcpyAsync(d + cnt, ux + off, cnt * sizeof(double), cudaMemcpyHostToDevice, L->copy_stream), "copying ux");
        OLB_CUDA(cudaMemcpyAsync(d + 2 * cnt, uy + off, cnt * sizeof(double), cudaMemcpyHostToDevice, L->copy_stream), "copying uy");
        OLB_CUDA(cudaEventRecord(L->ev_copy[b], L->copy_stream), "recording event");
        OLB_CUDA(cudaStreamWaitEvent(L->stream, L->ev_copy[b], 0), "ordering conversion");
        InitSpec s{};
        s.mode = INIT_FIELDS;
        s.rho = d;
        s.ux = d + cnt;
        s.uy = d + 2 * cnt;
        s.y0 = y0;
        s.rows = r;
        st = run_init(L, s);
        if (st != OLB_OK) return st;
        OLB_CUDA(cudaEventRecord(L->ev_main[b], L->stream), "recording event");
    }
    // the host arrays may be reused on return (every copy precedes a kernel
    // of the lattice stream)
    OLB_CUDA(cudaStreamSynchronize(L->stream), "synchronising field upload");
    return OLB_OK;
}

olb_status olb_step(olb_lattice *L, int64_t nsteps) {
    oreg::NvtxRange nvtx_("olb_step");
    olb_status st = check_lattice(L, true);
    if (st != OLB_OK) return st;
    if (L->batch) return fail(OLB_ERR_STATE, "lattice belongs to a batch: it advances with olb_batch_run");
    if (nsteps < 0) return fail(OLB_ERR_INVALID, "nsteps must be >= 0");
    StepArgs a{};
    a.nx = L->p.nx;
    a.ny = L->p.ny;
    a.pitch = L->pitch;
    a.plane = L->plane;
    a.passes = (int)warp_passes(L->pitch, L->p.ny, L->V);
    a.eq = kernel_eq(&L->p);
    a.coll = L->p.coll;
    a.layout = L->p.layout;
    a.comp = L->comp;
    a.sr = L->sr;
    a.walls = L->p.boundary == OLB_BOUNDARY_WALLS_X;
    a.warps_per_block = L->warps_per_block;
    // FP32 storage with the FP64 collision runs on the FP64 constants, whose
    // shifts are the FP32 storage's (make_const_f64_for)
    const bool c64 = L->f64_coll && L->p.storage == OLB_F32;
    a.kconst = L->p.storage == OLB_F64 || c64 ? static_cast<const void *>(&L->kd)
                                              : static_cast<const void *>(&L->kf);
    a.stream = L->stream;
    const size_t bytes = L->buf_elems * L->esize;
    char *mem = static_cast<char *>(L->mem);
    for (int64_t s = 0; s < nsteps; ++s) {
        a.parity = (int)(L->t & 1);
        a.t = L->t;
        if (L->p.layout == OLB_LAYOUT_AB) {
            a.src = mem + (size_t)(L->t & 1) * bytes;
            a.dst = mem + (size_t)((L->t + 1) & 1) * bytes;
        } else {
            a.src = mem;
            a.dst = nullptr;
        }
        cudaError_t e = c64 ? step_f32c64(a) : DISPATCH(L->p.storage, step, a);
        if (e != cudaSuccess) return cuda_fail(e, "launching stream-collide");
        L->t += 1;
    }
    return OLB_OK;
}

int64_t olb_time(const olb_lattice *L) { return L ? L->t : -1; }

olb_status olb_moments(olb_lattice *L, double *rho, double *ux, double *uy, double *theta_loc) {
    oreg::NvtxRange nvtx_("olb_moments");
    olb_status st = check_lattice(L, true);
    if (st != OLB_OK) return st;
    if (!rho || !ux || !uy) return fail(OLB_ERR_INVALID, "rho, ux, uy must not be NULL");
    // chunks alternate between the two halves of the scratch: the kernel of
    // chunk k (lattice stream) overlaps the copies of chunk k-1 (copy stream)
    const int rows = chunk_rows(L, 4);
    const size_t nx = L->p.nx, half = (size_t)rows * nx * 4;
    st = ensure_chunk(L, 2 * half * sizeof(double));
    if (st != OLB_OK) return st;
    st = ensure_pipeline(L);
    if (st != OLB_OK) return st;
    double *base = static_cast<double *>(L->d_chunk);
    StreamDrain drain_{L->stream}, drain_copy_{L->copy_stream};
    // kernels may write either half once the copy stream's earlier copies are done
    for (int b = 0; b < 2; ++b)
        OLB_CUDA(cudaEventRecord(L->ev_copy[b], L->copy_stream), "recording event");
    const StateGeom g = geom(L);
    for (int y0 = 0, k = 0; y0 < L->p.ny; y0 += rows, ++k) {
        const int b = k & 1;
        double *d = base + b * half;
        const int r = std::min(rows, L->p.ny - y0);
        const size_t cnt = (size_t)r * nx;
        double *dr = d, *dx = d + cnt, *dy = d + 2 * cnt, *dt = theta_loc ? d + 3 * cnt : nullptr;
        OLB_CUDA(cudaStreamWaitEvent(L->stream, L->ev_copy[b], 0), "ordering kernel");
        OLB_CUDA(DISPATCH(L->p.storage, moments, state_base(L), g, y0, r, L->kd, dr, dx, dy, dt,
                          L->stream),
                 "launching moments kernel");
        OLB_CUDA(cudaEventRecord(L->ev_main[b], L->stream), "recording event");
        OLB_CUDA(cudaStreamWaitEvent(L->copy_stream, L->ev_main[b], 0), "ordering copy");
        const size_t off = (size_t)y0 * nx;
        OLB_CUDA(cudaMemcpyAsync(rho + off, dr, cnt * sizeof(double), cudaMemcpyDeviceToHost, L->copy_stream), "copying rho");
        OLB_CUDA(cudaMemcpyAsync(ux + off, dx, cnt * sizeof(double), cudaMemcpyDeviceToHost, L->copy_stream), "copying ux");
        OLB_CUDA(cudaMemcpyAsync(uy + off, dy, cnt * sizeof(double), cudaMemcpyDeviceToHost, L->copy_stream), "copying uy");
        if (theta_loc)
            OLB_CUDA(cudaMemcpyAsync(theta_loc + off, dt, cnt * sizeof(double), cudaMemcpyDeviceToHost, L->copy_stream),
                     "copying theta");
        OLB_CUDA(cudaEventRecord(L->ev_copy[b], L->copy_stream), "recording event");
    }
    // the scratch is reused by later calls on the lattice stream: order it
    // after these copies; the host arrays are complete once the copy stream is
    OLB_CUDA(cudaStreamWaitEvent(L->stream, L->ev_copy[0], 0), "ordering scratch reuse");
    OLB_CUDA(cudaStreamWaitEvent(L->stream, L->ev_copy[1], 0), "ordering scratch reuse");
    OLB_CUDA(cudaStreamSynchronize(L->copy_stream), "synchronising moments");
    return OLB_OK;
}

olb_status olb_moments_device(olb_lattice *L, double *d_rho, double *d_ux, double *d_uy,
                              double *d_theta_loc) {
    olb_status st = check_lattice(L, true);
    if (st != OLB_OK) return st;
    if (!d_rho) return fail(OLB_ERR_INVALID, "d_rho must not be NULL");
    OLB_CUDA(DISPATCH(L->p.storage, moments, state_base(L), geom(L), 0, L->p.ny, L->kd, d_rho,
                      d_ux, d_uy, d_theta_loc, L->stream),
             "launching moments kernel");
    return OLB_OK;
}

olb_status olb_get_populations(olb_lattice *L, double *f9) {
    oreg::NvtxRange nvtx_("olb_get_populations");
    olb_status st = check_lattice(L, true);
    if (st != OLB_OK) return st;
    if (!f9) return fail(OLB_ERR_INVALID, "f9 must not be NULL");
    const int rows = chunk_rows(L, 9);
    const size_t nx = L->p.nx, N = nx * L->p.ny;
    st = ensure_chunk(L, (size_t)rows * nx * 9 * sizeof(double));
    if (st != OLB_OK) return st;
    double *d = static_cast<double *>(L->d_chunk);
    StreamDrain drain_{L->stream};
    const StateGeom g = geom(L);
    for (int y0 = 0; y0 < L->p.ny; y0 += rows) {
        const int r = std::min(rows, L->p.ny - y0);
        const size_t cnt = (size_t)r * nx;
        OLB_CUDA(DISPATCH(L->p.storage, get_canonical, state_base(L), g, 0, y0, L->p.nx, r, L->kd, d,
                          L->stream),
                 "launching population readback");
        for (int i = 0; i < 9; ++i)
            OLB_CUDA(cudaMemcpyAsync(f9 + i * N + (size_t)y0 * nx, d + i * cnt, cnt * sizeof(double),
                                     cudaMemcpyDeviceToHost, L->stream),
                     "copying populations");
        // scratch reuse by the next chunk is ordered by the stream
    }
    OLB_CUDA(cudaStreamSynchronize(L->stream), "synchronising population readback");
    return OLB_OK;
}

olb_status olb_get_region(olb_lattice *L, int32_t x0, int32_t y0, int32_t wx, int32_t wy,
                          double *f9) {
    olb_status st = check_lattice(L, true);
    if (st != OLB_OK) return st;
    if (!f9) return fail(OLB_ERR_INVALID, "f9 must not be NULL");
    if (x0 < 0 || y0 < 0 || wx < 1 || wy < 1 || (int64_t)x0 + wx > L->p.nx ||
        (int64_t)y0 + wy > L->p.ny)
        return fail(OLB_ERR_INVALID, "window [%d,+%d) x [%d,+%d) outside the %d x %d lattice", x0, wx,
                    y0, wy, L->p.nx, L->p.ny);
    const size_t row_bytes = (size_t)wx * 9 * sizeof(double);
    int rows = (int)std::max<size_t>(1, std::min<size_t>(CHUNK_BYTES_MAX / row_bytes, (size_t)wy));
    st = ensure_chunk(L, (size_t)rows * row_bytes);
    if (st != OLB_OK) return st;
    double *d = static_cast<double *>(L->d_chunk);
    StreamDrain drain_{L->stream};
    const StateGeom g = geom(L);
    const size_t W = (size_t)wx * wy;
    for (int r0 = 0; r0 < wy; r0 += rows) {
        const int r = std::min(rows, wy - r0);
        const size_t cnt = (size_t)r * wx;
        OLB_CUDA(DISPATCH(L->p.storage, get_canonical, state_base(L), g, x0, y0 + r0, wx, r, L->kd,
                          d, L->stream),
                 "launching region readback");
        for (int i = 0; i < 9; ++i)
            OLB_CUDA(cudaMemcpyAsync(f9 + i * W + (size_t)r0 * wx, d + i * cnt, cnt * sizeof(double),
                                     cudaMemcpyDeviceToHost, L->stream),
                     "copying region");
        // scratch reuse by the next chunk is ordered by the stream
    }
    OLB_CUDA(cudaStreamSynchronize(L->stream), "synchronising region readback");
    return OLB_OK;
}

olb_status olb_set_populations(olb_lattice *L, const double *f9, int64_t t) {
    oreg::NvtxRange nvtx_("olb_set_populations");
    olb_status st = check_lattice(L, false);
    if (st != OLB_OK) return st;
    if (!f9) return fail(OLB_ERR_INVALID, "f9 must not be NULL");
    if (t < 0) return fail(OLB_ERR_INVALID, "t must be >= 0");
    const int rows = chunk_rows(L, 9);
    const size_t nx = L->p.nx, N = nx * L->p.ny;
    st = ensure_chunk(L, (size_t)rows * nx * 9 * sizeof(double));
    if (st != OLB_OK) return st;
    L->t = t;
    double *d = static_cast<double *>(L->d_chunk);
    StreamDrain drain_{L->stream};
    const StateGeom g = geom(L);
    for (int y0 = 0; y0 < L->p.ny; y0 += rows) {
        const int r = std::min(rows, L->p.ny - y0);
        const size_t cnt = (size_t)r * nx;
        for (int i = 0; i < 9; ++i)
            OLB_CUDA(cudaMemcpyAsync(d + i * cnt, f9 + i * N + (size_t)y0 * nx, cnt * sizeof(double),
                                     cudaMemcpyHostToDevice, L->stream),
                     "copying populations");
        OLB_CUDA(DISPATCH(L->p.storage, set_canonical, state_base(L), g, y0, r, L->kd, d, L->stream),
                 "launching population upload");
        // scratch reuse by the next chunk is ordered by the stream
    }
    OLB_CUDA(cudaStreamSynchronize(L->stream), "synchronising population upload");
    return OLB_OK;
}

olb_status olb_diagnostics(olb_lattice *L, double *mass, double *mom_x, double *mom_y,
                           int64_t *nonfinite) {
    oreg::NvtxRange nvtx_("olb_diagnostics");
    olb_status st = check_lattice(L, true);
    if (st != OLB_OK) return st;
    ModeSpec mode{};
    double r[RED_QUANTITIES];
    st = reduce(L, mode, r);
    if (st != OLB_OK) return st;
    if (mass) *mass = r[0];
    if (mom_x) *mom_x = r[1];
    if (mom_y) *mom_y = r[2];
    const int64_t nf = (int64_t)llround(r[3]);
    if (nonfinite) *nonfinite = nf;
    if (nf > 0) return fail(OLB_ERR_NONFINITE, "%lld nodes hold non-finite populations at t = %lld",
                            (long long)nf, (long long)L->t);
    return OLB_OK;
}

olb_status olb_wave_mode(olb_lattice *L, int32_t m, int32_t n, double *a_sin, double *a_cos) {
    oreg::NvtxRange nvtx_("olb_wave_mode");
    olb_status st = check_lattice(L, true);
    if (st != OLB_OK) return st;
    if (!a_sin && !a_cos) return fail(OLB_ERR_INVALID, "a_sin and a_cos must not both be NULL");
    if (m == 0 && n == 0) return fail(OLB_ERR_INVALID, "wave vector (m, n) must not be (0, 0)");
    ModeSpec mode{};
    mode.active = 1;
    mode.m = m;
    mode.n = n;
    const double kx = (double)m / L->p.nx, ky = (double)n / L->p.ny;
    const double nk = std::hypot(kx, ky);
    mode.ex = -ky / nk;
    mode.ey = kx / nk;
    st = mode_tables(L, m, n);
    if (st != OLB_OK) return st;
    mode.tab = L->d_tab;
    double r[RED_QUANTITIES];
    st = reduce(L, mode, r);
    if (st != OLB_OK) return st;
    const double scale = 2.0 / ((double)L->p.nx * L->p.ny);
    if (a_sin) *a_sin = scale * r[4];
    if (a_cos) *a_cos = scale * r[5];
    if (r[3] > 0) return fail(OLB_ERR_NONFINITE, "state holds non-finite populations");
    return OLB_OK;
}

olb_status olb_wave_amplitude(olb_lattice *L, int32_t m, int32_t n, double *amp) {
    if (!amp) return fail(OLB_ERR_INVALID, "amp must not be NULL");
    return olb_wave_mode(L, m, n, amp, nullptr);
}

olb_status olb_destroy(olb_lattice *L) {
    if (!L) return OLB_OK;
    olb_status st = OLB_OK;
    if (L->batch) st = olb_batch_remove(L->batch, L);
    if (L->stream) {
        cudaError_t e = cudaStreamSynchronize(L->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "synchronising before destroy");
    }
    if (L->own_mem && L->mem) cudaFree(L->mem);
    if (L->d_red) cudaFree(L->d_red);
    if (L->h_red) cudaFreeHost(L->h_red);
    if (L->copy_stream) {
        cudaStreamSynchronize(L->copy_stream);
        for (int b = 0; b < 2; ++b) {
            cudaEventDestroy(L->ev_main[b]);
            cudaEventDestroy(L->ev_copy[b]);
        }
        cudaStreamDestroy(L->copy_stream);
    }
    if (L->d_chunk) cudaFree(L->d_chunk);
    if (L->d_tab) cudaFree(L->d_tab);
    if (L->d_cmp) cudaFree(L->d_cmp);
    if (L->h_tab) cudaFreeHost(L->h_tab);
    if (L->stream != L->owned_stream && L->owned_stream) {
        cudaError_t e = cudaStreamSynchronize(L->owned_stream);
        if (e != cudaSuccess && st == OLB_OK) st = cuda_fail(e, "synchronising before destroy");
    }
    if (L->owned_stream) cudaStreamDestroy(L->owned_stream);
    delete L;
    return st;
}

const char *olb_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
