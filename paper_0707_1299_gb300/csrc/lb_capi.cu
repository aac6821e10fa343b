// lb_capi.cu -- the C ABI declared in include/lb.h: argument validation,
// ownership of device memory, host/device pointer handling, and the order
// of the kernels within a time step.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>

#include "../../include/lb.h"
#include "lb_internal.h"

namespace {

thread_local std::string g_create_err;

lb_status fail(lb_ctx* c, lb_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_err = msg;
    return s;
}

lb_status cuda_fail(lb_ctx* c, cudaError_t e, const char* where) {
    return fail(c, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(call, where)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Staging area for host pointers: a single grow-only device buffer.
lb_status ensure_stage(lb_ctx* c, size_t bytes) {
    if (bytes <= c->stage_bytes) return LB_OK;
    if (c->stage) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->stage);
        c->stage = nullptr;
        c->stage_bytes = 0;
    }
    LB_CUDA(cudaMalloc(&c->stage, bytes), "staging allocation");
    c->stage_bytes = bytes;
    return LB_OK;
}

// Resolve up to four pointer arguments: device pointers pass through, host
// inputs are copied into the staging area, host outputs get a staging slot
// (copied back by finish_outputs).
struct Arg {
    const void* user;
    size_t bytes;
    bool is_output;
    void* dev;       // what the kernels see
    bool staged;
};

lb_status resolve(lb_ctx* c, Arg* args, int nargs, bool* any_host) {
    size_t need = 0;
    *any_host = false;
    for (int i = 0; i < nargs; ++i) {
        args[i].staged = args[i].user && !is_device_ptr(args[i].user);
        if (args[i].staged) need += (args[i].bytes + 255) & ~(size_t)255;
        *any_host = *any_host || args[i].staged;
    }
    if (need) {
        lb_status s = ensure_stage(c, need);
        if (s != LB_OK) return s;
    }
    size_t off = 0;
    for (int i = 0; i < nargs; ++i) {
        if (!args[i].user) {
            args[i].dev = nullptr;
        } else if (!args[i].staged) {
            args[i].dev = const_cast<void*>(args[i].user);
        } else {
            args[i].dev = (char*)c->stage + off;
            off += (args[i].bytes + 255) & ~(size_t)255;
            if (!args[i].is_output && args[i].bytes)
                LB_CUDA(cudaMemcpyAsync(args[i].dev, args[i].user, args[i].bytes, cudaMemcpyHostToDevice, c->stream),
                        "host-to-device copy");
        }
    }
    return LB_OK;
}

lb_status finish(lb_ctx* c, Arg* args, int nargs, bool any_host) {
    for (int i = 0; i < nargs; ++i)
        if (args[i].staged && args[i].is_output && args[i].bytes)
            LB_CUDA(cudaMemcpyAsync(const_cast<void*>(args[i].user), args[i].dev, args[i].bytes, cudaMemcpyDeviceToHost,
                                    c->stream),
                    "device-to-host copy");
    if (any_host && !c->host_async) LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    return LB_OK;
}

lb_status grow_points(lb_ctx* c, int need) {
    if (need <= c->cap) return LB_OK;
    int cap = std::max(need, std::max(64, 2 * c->cap));
    double *pos = nullptr, *force = nullptr, *radius = nullptr;
    int* mobile = nullptr;
    cudaError_t e = cudaMalloc(&pos, sizeof(double) * 3 * cap);
    if (e == cudaSuccess) e = cudaMalloc(&force, sizeof(double) * 3 * cap);
    if (e == cudaSuccess) e = cudaMalloc(&radius, sizeof(double) * cap);
    if (e == cudaSuccess) e = cudaMalloc(&mobile, sizeof(int) * cap);
    if (e == cudaSuccess && c->npts) {
        e = cudaMemcpyAsync(pos, c->pos, sizeof(double) * 3 * c->npts, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(force, c->force, sizeof(double) * 3 * c->npts, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(radius, c->radius, sizeof(double) * c->npts, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(mobile, c->mobile, sizeof(int) * c->npts, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(pos);
        cudaFree(force);
        cudaFree(radius);
        cudaFree(mobile);
        return cuda_fail(c, e, "point arrays");
    }
    cudaFree(c->pos);
    cudaFree(c->force);
    cudaFree(c->radius);
    cudaFree(c->mobile);
    c->pos = pos;
    c->force = force;
    c->radius = radius;
    c->mobile = mobile;
    c->cap = cap;
    return LB_OK;
}

lb_status invalidate_field(lb_ctx* c) {
    c->fix_ok = false;
    if (!c->field_ready) return LB_OK;
    LB_CUDA(lbk::launch_clear_field(c), "clear force field");
    c->field_ready = false;
    return LB_OK;
}

// Cell order of the points (the work order of the spread and the
// interpolation): recomputed when the points change and, for moving
// colloids, every SORT_INTERVAL steps.  Correctness never depends on it.
constexpr int SORT_INTERVAL = 64;

// Per-point buffers (order, sort workspace, stencil rows),
// grown with the point capacity.
lb_status ensure_point_buffers(lb_ctx* c) {
    const size_t ws = lbk::sort_ws_ints(c->geom, c->npts);
    if ((size_t)c->npts <= c->pt_cap && ws <= c->sort_ws_ints) return LB_OK;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->order);
    cudaFree(c->sort_ws);
    cudaFree(c->stencil);
    c->order = nullptr;
    c->sort_ws = nullptr;
    c->stencil = nullptr;
    c->pt_cap = c->sort_ws_ints = 0;
    const size_t cap = std::max<size_t>((size_t)c->npts, (size_t)c->cap);
    const size_t wcap = lbk::sort_ws_ints(c->geom, (long long)cap);
    LB_CUDA(cudaMalloc(&c->order, sizeof(int) * cap), "point order");
    LB_CUDA(cudaMalloc(&c->sort_ws, sizeof(int) * wcap), "point order workspace");
    LB_CUDA(cudaMalloc(&c->stencil, lbk::arith_bytes(c->prec) * lbk::ST_W * cap), "stencil rows");
    c->pt_cap = cap;
    c->sort_ws_ints = wcap;
    c->order_stale = c->npts > 0;
    c->stencil_ready = false;
    return LB_OK;
}

lb_status ensure_field(lb_ctx* c) {
    if (c->field_ready || c->npts == 0) return LB_OK;
    lb_status s = ensure_point_buffers(c);
    if (s != LB_OK) return s;
    if (c->order_stale) {  // a few points are taken in their own order
        if (c->npts > lbk::SORT_MIN_POINTS) LB_CUDA(lbk::launch_sort_points(c), "point order kernels");
        c->order_stale = false;
        c->steps_since_sort = 0;
    }
    LB_CUDA(lbk::launch_spread(c), "spread kernel");  // writes the stencil rows too
    c->stencil_ready = true;
    c->field_ready = true;
    // fixed points keep this field: list its tiles once for the fix-up path
    if (c->n_mobile == 0) LB_CUDA(lbk::list_fixed_tiles(c), "tile list");
    else c->fix_ok = false;
    return LB_OK;
}

// Velocity field of the collide kernel (lattices with colloids).
lb_status ensure_vel(lb_ctx* c) {
    LB_CUDA(lbk::ensure_velocity_field(c), "velocity field");
    return LB_OK;
}

// Phase timing: an event recorded on the context's stream before and after
// the launches of one phase of a step.
enum { PH_SPREAD = 0, PH_COLLIDE, PH_POINTS, PH_SORT, PH_CORRECTION, PH_COUNT };

lb_status phase_event(lb_ctx* c, cudaEvent_t* ev) {
    if (!c->ev_free.empty()) {
        *ev = c->ev_free.back();
        c->ev_free.pop_back();
    } else {
        LB_CUDA(cudaEventCreate(ev), "timing event");
    }
    LB_CUDA(cudaEventRecord(*ev, c->stream), "timing event record");
    return LB_OK;
}

lb_status phase_begin(lb_ctx* c, int phase) {
    if (!c->phase_timing) return LB_OK;
    cudaEvent_t e;
    lb_status s = phase_event(c, &e);
    if (s != LB_OK) return s;
    c->mark_phase.push_back(phase);
    c->mark_ev.push_back(e);
    return LB_OK;
}

lb_status phase_end(lb_ctx* c) {
    if (!c->phase_timing) return LB_OK;
    cudaEvent_t e;
    lb_status s = phase_event(c, &e);
    if (s == LB_OK) c->mark_ev.push_back(e);
    return s;
}

void drop_phase_events(lb_ctx* c) {
    for (cudaEvent_t e : c->mark_ev) c->ev_free.push_back(e);
    c->mark_ev.clear();
    c->mark_phase.clear();
}

}  // namespace

extern "C" {

lb_status lb_create(lb_ctx** out, const int grid[3], double tau_shear, double tau_bulk, int precision, void* stream) {
    lb_ctx* c = nullptr;
    if (!out) return fail(nullptr, LB_ERR_ARG, "lb_create: out is NULL");
    *out = nullptr;
    if (!grid) return fail(nullptr, LB_ERR_ARG, "lb_create: grid is NULL");
    for (int a = 0; a < 3; ++a)
        if (grid[a] < 1) return fail(nullptr, LB_ERR_ARG, "lb_create: grid sizes must be >= 1");
    const long long V = (long long)grid[0] * grid[1] * grid[2];
    if (V >= (1LL << 32)) return fail(nullptr, LB_ERR_ARG, "lb_create: lattice too large (nx*ny*nz >= 2^32)");
    if (!(tau_shear > 0) || !(tau_bulk > 0) || !isfinite(tau_shear) || !isfinite(tau_bulk))
        return fail(nullptr, LB_ERR_ARG, "lb_create: relaxation times must be finite and > 0");
    if (precision < LB_F64 || precision > LB_BF16S) return fail(nullptr, LB_ERR_ARG, "lb_create: unknown precision");

    c = new (std::nothrow) lb_ctx();
    if (c) {  // spreading of the point phase: direct global reductions, or staged in shared memory
        const char* sp = getenv("GB300LB_SPREAD");
        c->spread_shared = sp && strcmp(sp, "shared") == 0;
    }
    if (!c) return fail(nullptr, LB_ERR_OOM, "lb_create: host allocation failed");
    c->prec = precision;
    c->tau_s = tau_shear;
    c->tau_b = tau_bulk;
    c->g[0] = c->g[1] = c->g[2] = 0.0;
    c->counter = 1;
    c->a_L = INFINITY;
    c->seed = 0x2545F491u;
    c->scale = c->inv_scale = 1.0f;
    if (precision == LB_F16S) {
        c->scale = 1048576.0f;  // 2^20
        c->inv_scale = 1.0f / 1048576.0f;
    }
    c->stream = (cudaStream_t)stream;
    c->geom.nx = grid[0];
    c->geom.ny = grid[1];
    c->geom.nz = grid[2];
    c->geom.ntx = (grid[0] + lbk::TILE_X - 1) / lbk::TILE_X;
    c->geom.V = V;
    c->geom.ntiles = (long long)c->geom.ntx * grid[1] * grid[2];
    c->geom.wall_lo = c->geom.wall_hi = -1;
    c->geom.plane = (unsigned)grid[0] * (unsigned)grid[1];

    cudaError_t e = cudaGetDevice(&c->device);
    const size_t sb = lbk::storage_bytes(precision), ab = lbk::arith_bytes(precision);
    if (e == cudaSuccess) e = cudaMalloc(&c->f[0], sb * lbk::NQ * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&c->f[1], sb * lbk::NQ * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&c->floc, ab * lbk::FIELD_W * (size_t)V);
    if (e == cudaSuccess) e = cudaMalloc(&c->flags, sizeof(unsigned) * (size_t)c->geom.ntiles);  // 4 group flags a tile
    if (e == cudaSuccess) e = cudaMalloc(&c->fsum, sizeof(double) * 3);
    if (e == cudaSuccess) e = cudaMalloc(&c->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->partials, sizeof(double) * 4 * (size_t)lbk::moment_blocks(c->geom));
    if (e == cudaSuccess) e = cudaMalloc(&c->totals_dev, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->f[0], 0, sb * lbk::NQ * (size_t)V, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->floc, 0, ab * lbk::FIELD_W * (size_t)V, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, sizeof(unsigned) * (size_t)c->geom.ntiles, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->fsum, 0, sizeof(double) * 3, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lb_status s = fail(nullptr, e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA,
                           std::string("lb_create: ") + cudaGetErrorString(e));
        lb_destroy(c);
        return s;
    }
    lb_status s = grow_points(c, 64);
    if (s != LB_OK) {
        g_create_err = c->err;
        lb_destroy(c);
        return s;
    }
    *out = c;
    return LB_OK;
}

void lb_destroy(lb_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    cudaFree(c->f[0]);
    cudaFree(c->f[1]);
    cudaFree(c->floc);
    cudaFree(c->flags);
    cudaFree(c->vel);
    cudaFree(c->order);
    cudaFree(c->sort_ws);
    cudaFree(c->stencil);
    cudaFree(c->fix_list);
    cudaFree(c->pos);
    cudaFree(c->force);
    cudaFree(c->radius);
    cudaFree(c->mobile);
    cudaFree(c->fsum);
    cudaFree(c->status);
    cudaFree(c->partials);
    cudaFree(c->totals_dev);
    cudaFree(c->stage);
    cudaFree(c->corr_feat);
    cudaFree(c->corr_y);
    cudaFree(c->corr_ws);
    drop_phase_events(c);
    for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
    delete c;
}

const char* lb_last_error(const lb_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

lb_status lb_set_body_force(lb_ctx* c, const double g[3]) {
    if (!c) return LB_ERR_ARG;
    if (!g) return fail(c, LB_ERR_ARG, "lb_set_body_force: g is NULL");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(g[a])) return fail(c, LB_ERR_NONFINITE, "lb_set_body_force: non-finite g");
    for (int a = 0; a < 3; ++a) c->g[a] = g[a];
    c->version++;
    return LB_OK;
}

lb_status lb_set_walls_z(lb_ctx* c, int z_lo, int z_hi) {
    if (!c) return LB_ERR_ARG;
    if (z_lo < -1 || z_lo >= c->geom.nz || z_hi < -1 || z_hi >= c->geom.nz)
        return fail(c, LB_ERR_ARG, "lb_set_walls_z: plane outside the lattice");
    lb_status s = invalidate_field(c);
    if (s != LB_OK) return s;
    c->geom.wall_lo = z_lo;
    c->geom.wall_hi = z_hi;
    c->version++;
    return LB_OK;
}

lb_status lb_set_counterforce(lb_ctx* c, int enabled) {
    if (!c) return LB_ERR_ARG;
    c->counter = enabled ? 1 : 0;
    c->version++;
    return LB_OK;
}

lb_status lb_set_colloid_aL(lb_ctx* c, double a_L) {
    if (!c) return LB_ERR_ARG;
    if (!(a_L > 0) || isnan(a_L)) return fail(c, LB_ERR_ARG, "lb_set_colloid_aL: a_L must be > 0");
    c->a_L = a_L;
    c->version++;
    return LB_OK;
}

lb_status lb_add_point_forces(lb_ctx* c, int n, const double* pos, const double* F, int kind, const double* param) {
    if (!c) return LB_ERR_ARG;
    if (n < 0) return fail(c, LB_ERR_ARG, "lb_add_point_forces: n < 0");
    if (n == 0) return LB_OK;
    if (!pos || !F) return fail(c, LB_ERR_ARG, "lb_add_point_forces: pos or F is NULL");
    if (kind < LB_STOKESLET || kind > LB_COLLOID) return fail(c, LB_ERR_ARG, "lb_add_point_forces: unknown kind");
    if (kind != LB_STOKESLET && !param) return fail(c, LB_ERR_ARG, "lb_add_point_forces: param is required");
    const int mult = kind == LB_STRESSLET ? 2 : kind == LB_ROTLET ? 4 : 1;
    const long long total = (long long)c->npts + (long long)n * mult;
    if (total >= (1LL << 31) / 64) return fail(c, LB_ERR_ARG, "lb_add_point_forces: too many points");
    lb_status s = invalidate_field(c);
    if (s == LB_OK) s = grow_points(c, (int)total);
    if (s != LB_OK) return s;
    Arg args[3] = {{pos, sizeof(double) * 3 * n, false, nullptr, false},
                   {F, sizeof(double) * 3 * n, false, nullptr, false},
                   {param, param ? sizeof(double) * n : 0, false, nullptr, false}};
    bool any_host;
    s = resolve(c, args, 3, &any_host);
    if (s != LB_OK) return s;
    LB_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "status reset");
    LB_CUDA(lbk::launch_expand(c, n, (const double*)args[0].dev, (const double*)args[1].dev,
                               (const double*)args[2].dev, kind, mult),
            "expand kernel");
    int status = 0;
    LB_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status read");
    LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    if (status & 1) return fail(c, LB_ERR_NONFINITE, "lb_add_point_forces: non-finite position, force or parameter");
    if (status & 2)
        return fail(c, LB_ERR_ARG, "lb_add_point_forces: parameter must be > 0 (and |F| > 0 for stresslet/rotlet)");
    c->npts = (int)total;
    c->version++;
    c->order_stale = true;
    c->stencil_ready = false;
    if (kind == LB_COLLOID) c->n_mobile += n;
    LB_CUDA(lbk::launch_fsum(c), "force sum");
    LB_CUDA(cudaMemcpyAsync(c->fsum_host, c->fsum, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream),
            "force sum read");
    LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    return LB_OK;
}

lb_status lb_clear_point_forces(lb_ctx* c) {
    if (!c) return LB_ERR_ARG;
    lb_status s = invalidate_field(c);
    if (s != LB_OK) return s;
    c->npts = 0;
    c->n_mobile = 0;
    c->version++;
    for (int a = 0; a < 3; ++a) c->fsum_host[a] = 0.0;
    LB_CUDA(cudaMemsetAsync(c->fsum, 0, sizeof(double) * 3, c->stream), "force sum reset");
    return LB_OK;
}

lb_status lb_num_points(const lb_ctx* c, int* n_out) {
    if (!c || !n_out) return LB_ERR_ARG;
    *n_out = c->npts;
    return LB_OK;
}

lb_status lb_set_host_async(lb_ctx* c, int on) {
    if (!c) return LB_ERR_ARG;
    c->host_async = on != 0;
    return LB_OK;
}

// Whether all n values are finite: x - x is +0 for a finite x and NaN for
// an infinity or a NaN (IEEE arithmetic; the library is not built with
// value-changing floating-point options), summed in four independent
// chains: twice as fast as an early-exit test of each value.
static bool all_finite(const double* p, long long n) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    const long long m = n - n % 4;
    for (long long i = 0; i < m; i += 4)
        for (int k = 0; k < 4; ++k) a[k] += p[i + k] - p[i + k];
    for (long long i = m; i < n; ++i) a[0] += p[i] - p[i];
    return (a[0] + a[1]) + (a[2] + a[3]) == 0.0;
}

lb_status lb_set_positions(lb_ctx* c, const double* pos) {
    if (!c) return LB_ERR_ARG;
    if (c->npts == 0) return LB_OK;
    if (!pos) return fail(c, LB_ERR_ARG, "lb_set_positions: pos is NULL");
    // The update is all or nothing.  Device positions are checked by a
    // kernel whose result is read before anything changes.  Host positions
    // are checked on the host (the call need not wait for the device) while
    // the clear of the old field and the copy in run on the device: a
    // rejected update leaves the positions as they were, and the cleared
    // field is spread again where it is next needed.
    const bool on_device = is_device_ptr(pos);
    if (on_device) {
        LB_CUDA(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream), "status reset");
        LB_CUDA(lbk::launch_set_positions(c, pos, true), "position check kernel");
        int status = 0;
        LB_CUDA(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status read");
        LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
        if (status) return fail(c, LB_ERR_NONFINITE, "lb_set_positions: non-finite position");
    }
    lb_status s = invalidate_field(c);
    if (s != LB_OK) return s;
    Arg args[1] = {{pos, sizeof(double) * 3 * c->npts, false, nullptr, false}};
    bool any_host;
    s = resolve(c, args, 1, &any_host);
    if (s != LB_OK) return s;
    const bool finite = on_device || all_finite(pos, 3LL * c->npts);
    if (finite) LB_CUDA(lbk::launch_set_positions(c, (const double*)args[0].dev, false), "position kernel");
    // a host buffer is read by the time the call returns, unless host-async
    if (any_host && !c->host_async) LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    if (!finite) return fail(c, LB_ERR_NONFINITE, "lb_set_positions: non-finite position");
    c->order_stale = true;
    c->stencil_ready = false;
    return LB_OK;
}

namespace {
// Buffers of the learned correction and its candidate lists.
lb_status ensure_corr_buffers(lb_ctx* c) {
    const int box[3] = {c->geom.nx, c->geom.ny, c->geom.nz};
    if ((size_t)c->npts > c->corr_cap) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->corr_feat);
        cudaFree(c->corr_y);
        c->corr_feat = nullptr;
        c->corr_y = nullptr;
        c->corr_cap = 0;
        const size_t n = (size_t)c->npts;
        LB_CUDA(cudaMalloc(&c->corr_feat, sizeof(float) * 27 * n), "correction buffers");
        LB_CUDA(cudaMalloc(&c->corr_y, sizeof(float) * 3 * n), "correction buffers");
        c->corr_cap = n;
    }
    const int slots = lbk::verlet_capacity(c->npts, box);
    const size_t ws = lbk::verlet_ws_bytes(c->npts, box, slots);
    bool fresh = c->corr_ws_n != c->npts || c->corr_ws_slots != slots;
    if (ws > c->corr_ws_bytes) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->corr_ws);
        c->corr_ws = nullptr;
        c->corr_ws_bytes = 0;
        LB_CUDA(cudaMalloc(&c->corr_ws, ws), "correction workspace");
        c->corr_ws_bytes = ws;
        fresh = true;
    }
    if (fresh) {  // a rebuild on the next step (the lists index the points)
        LB_CUDA(lbk::verlet_reset(c->corr_ws, c->npts, box, slots, c->stream), "correction workspace");
        c->corr_ws_n = c->npts;
        c->corr_ws_slots = slots;
    }
    return LB_OK;
}
}  // namespace

lb_status lb_set_colloid_correction(lb_ctx* c, lb_mlp* net) {
    if (!c) return LB_ERR_ARG;
    c->corr = net;
    c->version++;
    return LB_OK;
}

lb_status lb_step(lb_ctx* c, int nsteps) {
    if (!c) return LB_ERR_ARG;
    if (nsteps < 0) return fail(c, LB_ERR_ARG, "lb_step: nsteps < 0");
    if (c->corr && c->n_mobile > 0) {
        lb_status st = ensure_corr_buffers(c);
        if (st != LB_OK) return st;
    }
    {
        lb_status st = ensure_vel(c);
        if (st != LB_OK) return st;
    }
    const int box[3] = {c->geom.nx, c->geom.ny, c->geom.nz};
    // Step n (Sec. IV with forward Euler): spread F^n at R^n unless the
    // previous step (or a query) already did; collide and stream with F^n,
    // writing v^n = (j + F^n/2) / rho at the stencil nodes and zeroing the
    // consumed force; then the point phase: interpolate v^n at R^n, move the
    // colloids (plus the learned correction when a network is attached) and
    // spread F^{n+1} at R^{n+1} for the next step.  Fixed points alone keep
    // their field from step to step (no point phase).
#define LB_PHASE(call)                       \
    do {                                     \
        lb_status ps_ = (call);              \
        if (ps_ != LB_OK) return ps_;        \
    } while (0)
    for (int s = 0; s < nsteps; ++s) {
        LB_PHASE(phase_begin(c, PH_SPREAD));
        lb_status st = ensure_field(c);
        if (st != LB_OK) return st;
        if (c->n_mobile > 0) {
            // the point phase needs the per-point buffers and the stencil rows
            // of the current positions even where the field was spread
            // elsewhere (a batch step leaves it spread and the rows stale)
            st = ensure_point_buffers(c);
            if (st != LB_OK) return st;
            if (!c->stencil_ready) {
                LB_CUDA(lbk::launch_stencil(c), "stencil kernel");
                c->stencil_ready = true;
            }
        }
        LB_PHASE(phase_end(c));
        if (c->n_mobile > 0 && c->order_stale) {  // the point phase's work order
            LB_PHASE(phase_begin(c, PH_SORT));
            if (c->npts > lbk::SORT_MIN_POINTS) LB_CUDA(lbk::launch_sort_points(c), "point order kernels");
            c->order_stale = false;
            c->steps_since_sort = 0;
            LB_PHASE(phase_end(c));
        }
        const bool corrected = c->n_mobile > 0 && c->corr;
        if (corrected) {
            // the network's inputs depend on R^n only.  (They do not depend
            // on the collide either, but run beside it on a second stream
            // they slow the bandwidth-bound collide by about as much as they
            // hide: in series on the one stream.)
            LB_PHASE(phase_begin(c, PH_CORRECTION));
            LB_CUDA(lbk::verlet_features(c->corr_ws, c->npts, c->corr_ws_slots, c->pos, box, c->corr_feat, c->stream),
                    "feature kernels");
            LB_CUDA(lbk::mlp_forward(c->corr, c->npts, c->corr_feat, c->corr_y, c->stream), "forward kernel");
            c->launches += lbk::MLP_FEATURE_LAUNCHES + 1;
            LB_PHASE(phase_end(c));
        }
        LB_PHASE(phase_begin(c, PH_COLLIDE));
        LB_CUDA(lbk::launch_collide(c), "collide-stream kernel");
        LB_PHASE(phase_end(c));
        c->cur ^= 1;
        if (c->n_mobile > 0) {
            LB_PHASE(phase_begin(c, PH_POINTS));
            LB_CUDA(lbk::launch_points(c, corrected ? c->corr_y : nullptr), "point kernel");
            LB_PHASE(phase_end(c));
            c->field_ready = true;  // the forces at the new positions, spread for the next step
            c->stencil_ready = true;
            if (++c->steps_since_sort >= SORT_INTERVAL) c->order_stale = true;
        }
    }
#undef LB_PHASE
    return LB_OK;
}

lb_status lb_velocity_at(lb_ctx* c, int n, const double* pos, double* v_out) {
    if (!c) return LB_ERR_ARG;
    if (n < 0) return fail(c, LB_ERR_ARG, "lb_velocity_at: n < 0");
    if (n == 0) return LB_OK;
    if (!pos || !v_out) return fail(c, LB_ERR_ARG, "lb_velocity_at: pos or v_out is NULL");
    Arg args[2] = {{pos, sizeof(double) * 3 * n, false, nullptr, false},
                   {v_out, sizeof(double) * 3 * n, true, nullptr, false}};
    bool any_host;
    lb_status s = resolve(c, args, 2, &any_host);
    if (s == LB_OK) s = ensure_field(c);
    if (s != LB_OK) return s;
    LB_CUDA(lbk::launch_gather(c, n, (const double*)args[0].dev, (double*)args[1].dev), "gather kernel");
    return finish(c, args, 2, any_host);
}

lb_status lb_colloid_velocity(lb_ctx* c, int n, const double* pos, const double* F, const double* radius,
                              double* U_out) {
    if (!c) return LB_ERR_ARG;
    if (n < 0) return fail(c, LB_ERR_ARG, "lb_colloid_velocity: n < 0");
    if (n == 0) return LB_OK;
    if (!pos || !F || !radius || !U_out) return fail(c, LB_ERR_ARG, "lb_colloid_velocity: NULL argument");
    Arg args[4] = {{pos, sizeof(double) * 3 * n, false, nullptr, false},
                   {F, sizeof(double) * 3 * n, false, nullptr, false},
                   {radius, sizeof(double) * n, false, nullptr, false},
                   {U_out, sizeof(double) * 3 * n, true, nullptr, false}};
    bool any_host;
    lb_status s = resolve(c, args, 4, &any_host);
    if (s == LB_OK) s = ensure_field(c);
    if (s != LB_OK) return s;
    LB_CUDA(lbk::launch_gather(c, n, (const double*)args[0].dev, (double*)args[3].dev), "gather kernel");
    LB_CUDA(lbk::launch_faxen(c, n, (const double*)args[1].dev, (const double*)args[2].dev, (double*)args[3].dev),
            "faxen kernel");
    return finish(c, args, 4, any_host);
}

lb_status lb_moments(lb_ctx* c, double* rho, double* u, double* totals) {
    if (!c) return LB_ERR_ARG;
    const size_t V = (size_t)c->geom.V;
    Arg args[3] = {{rho, sizeof(double) * V, true, nullptr, false},
                   {u, sizeof(double) * 3 * V, true, nullptr, false},
                   {totals, sizeof(double) * 4, true, nullptr, false}};
    bool any_host;
    lb_status s = resolve(c, args, 3, &any_host);
    if (s == LB_OK) s = ensure_field(c);
    if (s != LB_OK) return s;
    LB_CUDA(lbk::launch_moments(c, (double*)args[0].dev, (double*)args[1].dev, totals != nullptr), "moments kernel");
    if (totals)
        LB_CUDA(cudaMemcpyAsync(args[2].dev, c->totals_dev, sizeof(double) * 4, cudaMemcpyDeviceToDevice, c->stream),
                "totals copy");
    return finish(c, args, 3, any_host);
}

lb_status lb_particles(lb_ctx* c, double* pos_out, double* f_out) {
    if (!c) return LB_ERR_ARG;
    const size_t b = sizeof(double) * 3 * (size_t)c->npts;
    Arg args[2] = {{pos_out, b, true, nullptr, false}, {f_out, b, true, nullptr, false}};
    bool any_host;
    lb_status s = resolve(c, args, 2, &any_host);
    if (s != LB_OK) return s;
    if (pos_out && b)
        LB_CUDA(cudaMemcpyAsync(args[0].dev, c->pos, b, cudaMemcpyDeviceToDevice, c->stream), "position copy");
    if (f_out && b)
        LB_CUDA(cudaMemcpyAsync(args[1].dev, c->force, b, cudaMemcpyDeviceToDevice, c->stream), "force copy");
    return finish(c, args, 2, any_host);
}

lb_status lb_get_populations(lb_ctx* c, double* df) {
    if (!c) return LB_ERR_ARG;
    if (!df) return fail(c, LB_ERR_ARG, "lb_get_populations: df is NULL");
    Arg args[1] = {{df, sizeof(double) * lbk::NQ * (size_t)c->geom.V, true, nullptr, false}};
    bool any_host;
    lb_status s = resolve(c, args, 1, &any_host);
    if (s != LB_OK) return s;
    LB_CUDA(lbk::launch_convert_out(c, (double*)args[0].dev), "convert kernel");
    return finish(c, args, 1, any_host);
}

lb_status lb_set_populations(lb_ctx* c, const double* df) {
    if (!c) return LB_ERR_ARG;
    if (!df) return fail(c, LB_ERR_ARG, "lb_set_populations: df is NULL");
    Arg args[1] = {{df, sizeof(double) * lbk::NQ * (size_t)c->geom.V, false, nullptr, false}};
    bool any_host;
    lb_status s = resolve(c, args, 1, &any_host);
    if (s != LB_OK) return s;
    LB_CUDA(lbk::launch_convert_in(c, (const double*)args[0].dev), "convert kernel");
    return finish(c, args, 1, any_host);
}

// ------------------------------------------------------------ checkpoints
// File layout (host byte order): a fixed header, then the expanded point
// arrays, then the populations of the current step in the storage format
// (raw bytes: a restart continues bit for bit), then a 64-bit FNV-1a hash
// of everything before it.
namespace {

struct CkptHeader {
    char magic[8];            // "LBCKPT1\0"
    int grid[3], prec;
    double tau_s, tau_b, g[3], a_L;
    int counter, wall_lo, wall_hi;
    unsigned seed;
    float scale, inv_scale;
    int npts, n_mobile;
    long long pop_bytes;
};

struct Fnv {
    unsigned long long h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    }
};

constexpr size_t CKPT_CHUNK = (size_t)64 << 20;

bool write_all(FILE* f, const void* p, size_t n, Fnv& h) {
    h.add(p, n);
    return fwrite(p, 1, n, f) == n;
}

bool read_all(FILE* f, void* p, size_t n, Fnv& h) {
    if (fread(p, 1, n, f) != n) return false;
    h.add(p, n);
    return true;
}

}  // namespace

lb_status lb_save(lb_ctx* c, const char* path) {
    if (!c) return LB_ERR_ARG;
    if (!path) return fail(c, LB_ERR_ARG, "lb_save: path is NULL");
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "LBCKPT1", 8);
    h.grid[0] = c->geom.nx;
    h.grid[1] = c->geom.ny;
    h.grid[2] = c->geom.nz;
    h.prec = c->prec;
    h.tau_s = c->tau_s;
    h.tau_b = c->tau_b;
    for (int a = 0; a < 3; ++a) h.g[a] = c->g[a];
    h.a_L = c->a_L;
    h.counter = c->counter;
    h.wall_lo = c->geom.wall_lo;
    h.wall_hi = c->geom.wall_hi;
    h.seed = c->seed;
    h.scale = c->scale;
    h.inv_scale = c->inv_scale;
    h.npts = c->npts;
    h.n_mobile = c->n_mobile;
    h.pop_bytes = (long long)(lbk::storage_bytes(c->prec) * lbk::NQ * (size_t)c->geom.V);
    const size_t n = (size_t)c->npts;
    std::string pts;
    pts.resize(n * (sizeof(double) * 7 + sizeof(int)));
    char* q = &pts[0];
    if (n) {
        LB_CUDA(cudaMemcpyAsync(q, c->pos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->stream), "copy");
        LB_CUDA(cudaMemcpyAsync(q + sizeof(double) * 3 * n, c->force, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                                c->stream),
                "copy");
        LB_CUDA(cudaMemcpyAsync(q + sizeof(double) * 6 * n, c->radius, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                c->stream),
                "copy");
        LB_CUDA(cudaMemcpyAsync(q + sizeof(double) * 7 * n, c->mobile, sizeof(int) * n, cudaMemcpyDeviceToHost,
                                c->stream),
                "copy");
    }
    LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(c, LB_ERR_ARG, std::string("lb_save: cannot open ") + path);
    Fnv hash;
    bool ok = write_all(f, &h, sizeof(h), hash) && write_all(f, pts.data(), pts.size(), hash);
    std::string buf;
    buf.resize(std::min<size_t>(CKPT_CHUNK, (size_t)h.pop_bytes));
    const char* src = (const char*)c->f[c->cur];
    for (size_t off = 0; ok && off < (size_t)h.pop_bytes; off += buf.size()) {
        const size_t len = std::min(buf.size(), (size_t)h.pop_bytes - off);
        cudaError_t e = cudaMemcpyAsync(&buf[0], src + off, len, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            fclose(f);
            return cuda_fail(c, e, "lb_save: population copy");
        }
        ok = write_all(f, buf.data(), len, hash);
    }
    const unsigned long long digest = hash.h;
    ok = ok && fwrite(&digest, sizeof(digest), 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(c, LB_ERR_ARG, std::string("lb_save: write failed: ") + path);
    return LB_OK;
}

lb_status lb_load(lb_ctx* c, const char* path) {
    if (!c) return LB_ERR_ARG;
    if (!path) return fail(c, LB_ERR_ARG, "lb_load: path is NULL");
    FILE* f = fopen(path, "rb");
    if (!f) return fail(c, LB_ERR_ARG, std::string("lb_load: cannot open ") + path);
    Fnv hash;
    CkptHeader h;
    const long long pop_bytes = (long long)(lbk::storage_bytes(c->prec) * lbk::NQ * (size_t)c->geom.V);
    if (!read_all(f, &h, sizeof(h), hash) || memcmp(h.magic, "LBCKPT1", 8) != 0) {
        fclose(f);
        return fail(c, LB_ERR_ARG, "lb_load: not a checkpoint file");
    }
    if (h.grid[0] != c->geom.nx || h.grid[1] != c->geom.ny || h.grid[2] != c->geom.nz || h.prec != c->prec ||
        h.pop_bytes != pop_bytes) {
        fclose(f);
        return fail(c, LB_ERR_ARG, "lb_load: checkpoint of another grid or precision");
    }
    // A file written by another build or tool can carry an intact digest
    // and still hold values that the kernels would index with: the header
    // and (below) the point block get the checks the setters apply.
    if (h.npts < 0 || (long long)h.npts >= (1LL << 31) / 64 || h.n_mobile < 0 || h.n_mobile > h.npts ||
        h.wall_lo < -1 || h.wall_lo >= c->geom.nz || h.wall_hi < -1 || h.wall_hi >= c->geom.nz ||
        !(h.tau_s > 0) || !(h.tau_b > 0) || !isfinite(h.tau_s) || !isfinite(h.tau_b) || !(h.a_L > 0) ||
        isnan(h.a_L) || !isfinite(h.g[0]) || !isfinite(h.g[1]) || !isfinite(h.g[2]) ||
        (h.counter != 0 && h.counter != 1) || h.scale != c->scale || h.inv_scale != c->inv_scale) {
        fclose(f);
        return fail(c, LB_ERR_ARG, "lb_load: checkpoint header out of range");
    }
    const size_t n = (size_t)h.npts;
    std::string pts;
    pts.resize(n * (sizeof(double) * 7 + sizeof(int)));
    std::string pops;
    pops.resize((size_t)pop_bytes);
    unsigned long long digest = 0;
    const bool ok = read_all(f, &pts[0], pts.size(), hash) && read_all(f, &pops[0], pops.size(), hash) &&
                    fread(&digest, sizeof(digest), 1, f) == 1 && digest == hash.h;
    fclose(f);
    if (!ok) return fail(c, LB_ERR_ARG, "lb_load: truncated or corrupt checkpoint");
    {  // positions finite and inside [0, n), forces finite, radius > 0 and mobile flag 1 for colloids only
        const double* P = (const double*)pts.data();
        const double* Fp = P + 3 * n;
        const double* Rd = P + 6 * n;
        int* Mb = (int*)(P + 7 * n);
        const int nn[3] = {c->geom.nx, c->geom.ny, c->geom.nz};
        int mobile = 0;
        for (size_t k = 0; k < n; ++k) {
            int mb;
            memcpy(&mb, Mb + k, sizeof(int));
            double rad;
            memcpy(&rad, Rd + k, sizeof(double));
            bool good = (mb == 0 || mb == 1) && isfinite(rad) && (mb ? rad > 0 : rad >= 0);
            for (int a = 0; a < 3 && good; ++a) {
                double x, F;
                memcpy(&x, P + 3 * k + a, sizeof(double));
                memcpy(&F, Fp + 3 * k + a, sizeof(double));
                good = isfinite(x) && x >= 0.0 && x < (double)nn[a] && isfinite(F);
            }
            if (!good) return fail(c, LB_ERR_ARG, "lb_load: checkpoint point block out of range");
            mobile += mb;
        }
        if (mobile != h.n_mobile) return fail(c, LB_ERR_ARG, "lb_load: checkpoint mobile count mismatch");
    }
    // the file is complete, intact and in range: replace the state
    lb_status s = invalidate_field(c);
    if (s == LB_OK) s = grow_points(c, std::max(h.npts, 1));
    if (s != LB_OK) return s;
    const char* q = pts.data();
    if (n) {
        LB_CUDA(cudaMemcpyAsync(c->pos, q, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream), "copy");
        LB_CUDA(cudaMemcpyAsync(c->force, q + sizeof(double) * 3 * n, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                                c->stream),
                "copy");
        LB_CUDA(cudaMemcpyAsync(c->radius, q + sizeof(double) * 6 * n, sizeof(double) * n, cudaMemcpyHostToDevice,
                                c->stream),
                "copy");
        LB_CUDA(cudaMemcpyAsync(c->mobile, q + sizeof(double) * 7 * n, sizeof(int) * n, cudaMemcpyHostToDevice,
                                c->stream),
                "copy");
    }
    LB_CUDA(cudaMemcpyAsync(c->f[c->cur], pops.data(), (size_t)pop_bytes, cudaMemcpyHostToDevice, c->stream),
            "population copy");
    c->tau_s = h.tau_s;
    c->tau_b = h.tau_b;
    for (int a = 0; a < 3; ++a) c->g[a] = h.g[a];
    c->a_L = h.a_L;
    c->counter = h.counter;
    c->geom.wall_lo = h.wall_lo;
    c->geom.wall_hi = h.wall_hi;
    c->seed = h.seed;
    c->scale = h.scale;
    c->inv_scale = h.inv_scale;
    c->npts = h.npts;
    c->n_mobile = h.n_mobile;
    c->order_stale = true;
    c->stencil_ready = false;
    c->version++;
    LB_CUDA(lbk::launch_fsum(c), "force sum");
    LB_CUDA(cudaMemcpyAsync(c->fsum_host, c->fsum, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream),
            "force sum read");
    LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    return LB_OK;
}

lb_status lb_set_phase_timing(lb_ctx* c, int on) {
    if (!c) return LB_ERR_ARG;
    c->phase_timing = on != 0;
    if (!c->phase_timing) {
        LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
        drop_phase_events(c);
    }
    return LB_OK;
}

lb_status lb_phase_times(lb_ctx* c, double ms[5], long long counts[5]) {
    if (!c || !ms) return LB_ERR_ARG;
    LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    for (int p = 0; p < PH_COUNT; ++p) {
        ms[p] = 0.0;
        if (counts) counts[p] = 0;
    }
    const size_t n = c->mark_phase.size();
    if (c->mark_ev.size() != 2 * n) {  // a step failed between a begin and its end
        drop_phase_events(c);
        return fail(c, LB_ERR_STATE, "lb_phase_times: unpaired timing events (a step failed)");
    }
    for (size_t k = 0; k < n; ++k) {
        float t = 0.0f;
        cudaError_t e = cudaEventElapsedTime(&t, c->mark_ev[2 * k], c->mark_ev[2 * k + 1]);
        if (e != cudaSuccess) {
            drop_phase_events(c);
            return cuda_fail(c, e, "timing event read");
        }
        ms[c->mark_phase[k]] += (double)t;
        if (counts) counts[c->mark_phase[k]]++;
    }
    drop_phase_events(c);
    return LB_OK;
}

lb_status lb_kernel_launches(const lb_ctx* c, long long* count) {
    if (!c || !count) return LB_ERR_ARG;
    *count = c->launches;
    return LB_OK;
}

lb_status lb_synchronize(lb_ctx* c) {
    if (!c) return LB_ERR_ARG;
    LB_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
    return LB_OK;
}

lb_status lb_compute_aL(const int grid[3], const double R[3], const double dir[3], double* a_L) {
    lb_ctx* c = nullptr;
    if (!grid || !R || !a_L) return fail(nullptr, LB_ERR_ARG, "lb_compute_aL: NULL argument");
    for (int a = 0; a < 3; ++a) {
        if (grid[a] < 1) return fail(nullptr, LB_ERR_ARG, "lb_compute_aL: grid sizes must be >= 1");
        if (!isfinite(R[a]) || (dir && !isfinite(dir[a])))
            return fail(nullptr, LB_ERR_NONFINITE, "lb_compute_aL: non-finite input");
    }
    if (dir && dir[0] == 0 && dir[1] == 0 && dir[2] == 0)
        return fail(nullptr, LB_ERR_ARG, "lb_compute_aL: zero direction");
    double inv = 0.0;
    LB_CUDA(lbk::compute_inv_aL(grid, R, dir, &inv), "lb_compute_aL");
    *a_L = inv > 0 ? 1.0 / inv : INFINITY;
    return LB_OK;
}

}  // extern "C"
