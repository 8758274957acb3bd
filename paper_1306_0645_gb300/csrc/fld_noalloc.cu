// fld_noalloc.cu -- fld_residual_noalloc: the FP64 residual r = b - A x
// with ||r||^2 and max |r|, for callers that must not allocate device
// memory.
//
// Who cannot allocate: code whose device memory is owned by someone else's
// allocator (a host application that hands this library a fixed pool and
// forbids raw cudaMalloc), and latency-critical loops where cudaMalloc /
// cudaFree may synchronise the device and stall for milliseconds.  The
// contexts of fld_create allocate their work buffers once; this entry point
// needs no context at all.
//
// The reduction's scratch (per-block partial sums, the arrival counter and
// the result slots) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and keeps it; make that first call before any stream
// capture.  All calls share the array and it keeps the last call's
// contents: each call clears the counter and result slots first, and calls
// that overlap on the GPU (two streams at once) race on it.
#include <mutex>
#include <string>

#include "fld.h"
#include "kernels.h"

namespace {

using namespace fld;

// Scratch layout (doubles): 2 x RED_MAX_BLOCKS partial sums, then the scalar
// slots, then one word holding the block-arrival counter.
constexpr size_t NOALLOC_PARTIALS = 2 * (size_t)RED_MAX_BLOCKS;
constexpr size_t NOALLOC_SLOTS = NUM_SLOTS;
constexpr size_t NOALLOC_WORDS = NOALLOC_PARTIALS + NOALLOC_SLOTS + 1;

static __device__ __align__(256) double g_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_lock;
double* g_scratch_addr[MAX_DEVICES] = {};

// message for fld_last_error (defined with the other entry points)
fld_status fail(fld_status st, const std::string& msg) {
    fld::record_error(msg.c_str());
    return st;
}

// Device address of g_scratch on the current device (set up once per device).
fld_status scratch_address(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(FLD_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(FLD_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_lock);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(FLD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return FLD_OK;
}

}  // namespace

extern "C" {

fld_status fld_residual_noalloc(const fld_grid* g, const double* m, const double* wx,
                                const double* wy, const double* wz, const double* b,
                                const double* x, double* r, double* norms, void* cuda_stream) {
    if (!g || !m || !wx || !wy || !wz || !b || !x || !norms)
        return fail(FLD_EINVAL, "fld_residual_noalloc: null argument");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return fail(FLD_EINVAL, "fld_residual_noalloc: grid dimensions must be >= 1");
    {
        char msg[160];
        if (!bc_valid(g, msg, sizeof msg)) return fail(FLD_EINVAL, std::string("fld_residual_noalloc: ") + msg);
    }
    Dims d;
    d.nx = g->nx;
    d.ny = g->ny;
    d.nz = g->nz;
    d.px = g->bc[0] == FLD_BC_PERIODIC;
    d.py = g->bc[1] == FLD_BC_PERIODIC;
    d.pz = g->bc[2] == FLD_BC_PERIODIC;
    d.n = (long long)d.nx * d.ny * d.nz;
    // the fixed scratch holds the partial sums of at most RED_MAX_BLOCKS
    // blocks, the most the launch of an x-y plane of about 2^22 cells needs
    const ColShape sh = residual64_shape(d);
    if ((long long)sh.grid.x * sh.grid.y * sh.grid.z > RED_MAX_BLOCKS || d.n > (1LL << 33))
        return fail(FLD_EINVAL,
                    "fld_residual_noalloc: grid too large for the fixed scratch (an x-y plane may need "
                    "at most 16384 thread blocks of 256 cells, about 4194304 cells; 2^33 cells in all)");
    double* scratch = nullptr;
    fld_status st = scratch_address(&scratch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* sc = scratch + NOALLOC_PARTIALS;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + NOALLOC_PARTIALS + NOALLOC_SLOTS);
    // what must start at zero: the result slots (the non-finite flag) and the
    // arrival counter
    cudaError_t e = cudaMemsetAsync(sc, 0, (NOALLOC_SLOTS + 1) * sizeof(double), s);
    if (e != cudaSuccess) return fail(FLD_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    Op<double> A;
    A.m = const_cast<double*>(m);
    A.wx = const_cast<double*>(wx);
    A.wy = const_cast<double*>(wy);
    A.wz = const_cast<double*>(wz);
    A.invd = nullptr;
    RedArgs ra;
    ra.partials = scratch;
    ra.counter = counter;
    ra.sc = sc;
    ra.op = R_STORE_SUM_MAX;
    ra.slot0 = S_TRUE_RR;
    ra.slot1 = S_RMAX;
    ra.first = 0;
    launch_residual64(d, A, nullptr, b, x, r, ra, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FLD_ECUDA, std::string("residual launch: ") + cudaGetErrorString(e));
    e = cudaMemcpyAsync(norms, sc + S_TRUE_RR, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(norms + 1, sc + S_RMAX, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(FLD_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    return FLD_OK;
}

}  // extern "C"
