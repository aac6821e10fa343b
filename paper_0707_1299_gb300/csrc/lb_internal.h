// lb_internal.h -- the context behind the C ABI and the kernel launchers
// shared by lb_kernels.cu and lb_capi.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lb_device.cuh"

struct lb_mlp;

struct lb_ctx {
    lbk::Geom geom;
    int prec;                 // lb_precision
    double tau_s, tau_b;
    double g[3];
    int counter;              // 1: uniform counter-force on
    double a_L;               // +inf: no subtraction
    float scale, inv_scale;   // storage scale of the half formats (1 otherwise)
    cudaStream_t stream;
    int device;

    void* f[2];               // population buffers (19 V elements of the storage type)
    int cur;                  // index of the buffer holding the current state
    void* floc;               // localised force field, FIELD_W V elements of the arithmetic type
                              // (x, y, z, unused per site)
    lbk::flag_t* flags;       // one byte per 8-site x-group (four per 32-site tile): the group
                              // holds spread force
    void* vel;                // fluid velocity in the flagged groups, FIELD_W V elements of the
                              // arithmetic type (lattices with colloids only)
    bool host_async;          // host-memory copies are not waited for (lb_set_host_async)
    bool field_ready;         // floc holds the forces at the current positions
    unsigned* fix_list;       // flagged tiles of a field of fixed points, then their count
    bool fix_ok;              // few fixed points, listed: collide field-free + fix-up

    // monopoles after expansion (device, xyz interleaved)
    int npts, cap, n_mobile;
    double* pos;
    double* force;
    double* radius;           // > 0 for colloids, 0 for fixed points
    int* mobile;
    double* fsum;             // 3 doubles: net point force (device)
    double fsum_host[3];      // its host copy, refreshed when the points change
    int* status;              // 1 int: device-side validation result
    // per-point work buffers of the spread and the point phase
    int* order;               // the points in cell order
    int* sort_ws;
    void* stencil;            // stencil rows (ST_W elements of the arithmetic type per point)
    size_t pt_cap, sort_ws_ints;
    bool order_stale;         // positions changed since the last sort
    bool stencil_ready;       // stencil rows match the positions
    int steps_since_sort;

    // reductions
    double* partials;         // 4 doubles per block of the moments kernel
    double* totals_dev;       // 4 doubles

    // staging for host pointers (grown on demand)
    void* stage;
    size_t stage_bytes;

    // learned correction of the colloid velocity (optional)
    lb_mlp* corr;
    float* corr_feat;         // features (27 npts)
    float* corr_y;            // network output (3 npts)
    void* corr_ws;            // candidate lists of the features (verlet_features)
    size_t corr_cap, corr_ws_bytes;
    long long corr_ws_n;      // points and list slots the lists were laid out for
    int corr_ws_slots;

    // phase timing (lb_set_phase_timing): an event pair around each phase of
    // every lb_step, summed by lb_phase_times
    bool phase_timing;
    std::vector<cudaEvent_t> ev_free;   // recorded and read back, ready for reuse
    std::vector<int> mark_phase;        // phase of each recorded pair
    std::vector<cudaEvent_t> mark_ev;   // start, end of each recorded pair

    int spread_shared;        // 1: the point phase stages its spread in shared memory (GB300LB_SPREAD)

    long long launches;       // kernels launched so far
    unsigned seed;            // seed of the stochastic rounding of the 16-bit formats
    unsigned version;         // bumped by every configuration change (batches check it)

    std::string err;
};

namespace lbk {

// Uniform force density on fluid sites (body force + counter-force), in
// the arithmetic type of the kernel.
template <typename T>
struct UForce {
    T F[3];
};

cudaError_t launch_collide(lb_ctx* c);
cudaError_t launch_spread(lb_ctx* c);  // stencil rows at the positions, and the spread there
cudaError_t launch_gather(lb_ctx* c, int n, const double* qpos, double* vout);
cudaError_t launch_points(lb_ctx* c, const float* y);
cudaError_t launch_stencil(lb_ctx* c);
constexpr int SORT_MIN_POINTS = 2048;  // fewer points are taken in their own order
cudaError_t launch_sort_points(lb_ctx* c);
cudaError_t ensure_velocity_field(lb_ctx* c);
cudaError_t list_fixed_tiles(lb_ctx* c);
size_t sort_ws_ints(const Geom& g, long long npts);
size_t scan_ws_ints(long long m);
cudaError_t scan_exclusive(const int* in, long long m, int* out, int* bsum, cudaStream_t st);
cudaError_t launch_moments(lb_ctx* c, double* rho, double* u, bool want_totals);
cudaError_t launch_expand(lb_ctx* c, int n, const double* pos, const double* F, const double* param, int kind,
                          int mult);
cudaError_t launch_fsum(lb_ctx* c);
cudaError_t launch_faxen(lb_ctx* c, int n, const double* F, const double* a, double* U);
// check: only test pos (device) for non-finite values into c->status; else
// copy the checked positions in, wrapped into the box.
cudaError_t launch_set_positions(lb_ctx* c, const double* pos, bool check);
cudaError_t launch_convert_out(lb_ctx* c, double* df);
cudaError_t launch_convert_in(lb_ctx* c, const double* df);
cudaError_t launch_clear_field(lb_ctx* c);
template <typename T>
UForce<T> uniform_force(const lb_ctx* c);
constexpr int MLP_FEATURE_LAUNCHES = 6;  // kernels of one mlp_features or verlet_features call
size_t mlp_features_ws_ints(long long n, const int box[3]);
cudaError_t mlp_features(long long n, const double* pos, const int box[3], float* feat, int* ws, cudaStream_t st);
// Features of a lattice's colloids with candidate lists kept between steps
// (rebuilt on the device when a point has moved too far): list slots per
// point, workspace bytes, reset (forces a rebuild), and the feature call.
int verlet_capacity(long long n, const int box[3]);
size_t verlet_ws_bytes(long long n, const int box[3], int cap);
cudaError_t verlet_reset(void* ws, long long n, const int box[3], int cap, cudaStream_t st);
cudaError_t verlet_features(void* ws, long long n, int cap, const double* pos, const int box[3], float* feat,
                            cudaStream_t st);
cudaError_t mlp_forward(const lb_mlp* net, long long n, const float* feat, float* out, cudaStream_t st);
cudaError_t compute_inv_aL(const int grid[3], const double R[3], const double dir[3], double* inv_aL);

// ------------------------------------------------- shared launch helpers
constexpr int CS_WARPS = 4;  // tiles (warps) per block of the site kernels
constexpr int CS_THREADS = CS_WARPS * 32;

inline bool has_walls(const lb_ctx* c) { return c->geom.wall_lo >= 0 || c->geom.wall_hi >= 0; }
inline dim3 site_block() { return dim3(TILE_X, CS_WARPS, 1); }
// Capacity of the fixed-point tile list: 1/64 of all tiles, at least 1024.
inline unsigned fixed_tile_cap(const lb_ctx* c) {
    return (unsigned)std::max<long long>(1024, c->geom.ntiles / 64);
}

template <typename S>
inline Pops<S> pops(void* base, long long V) {
    Pops<S> p;
    for (int i = 0; i < NQ; ++i) p.p[i] = (S*)base + (size_t)i * (size_t)V;
    return p;
}

// Site kernels: block = 4 warps, one warp per 32-site x-row tile; grid =
// (tiles per row, ceil(ny / 4), nz).  No division in the index math.
inline dim3 site_grid(const Geom& g) {
    return dim3((unsigned)g.ntx, (unsigned)((g.ny + CS_WARPS - 1) / CS_WARPS), (unsigned)g.nz);
}

size_t storage_bytes(int prec);
size_t arith_bytes(int prec);
long long moment_blocks(const Geom& g);

}  // namespace lbk
