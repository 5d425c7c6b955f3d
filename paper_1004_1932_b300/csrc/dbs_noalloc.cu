// dbs_mobility_apply_noalloc: the mobility product v = H F for caller-owned
// device buffers, with every piece of scratch memory in a fixed array that is
// part of the library image, so that the call never allocates.
//
// Who needs this: callers that must not (or cannot) call cudaMalloc while they
// run -- a host framework that owns all device memory through its own capped
// pool, a plugin running inside such a framework, or a latency-critical loop
// where cudaMalloc/cudaFree would stall the device.  The handle-based API
// allocates its buffers at dbs_create_suspension; this entry point needs no
// handle and allocates nothing.
//
// The scratch array is shared by every call in the process on a given GPU, and
// it keeps the contents of the last call: calls that overlap on the GPU (for
// example on two streams at once) race on it and must be serialised by the
// caller.  The first call on a device resolves the array's device address with
// cudaGetSymbolAddress (a one-time set-up per device); make that first call
// before any stream capture.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "dbs.h"
#include "dbs_common.cuh"
#include "eval_kernel.cuh"

using namespace dbs;

namespace {

constexpr int NA_BT = 32;          // dumbbells per CTA (the small-system configuration)
constexpr int NA_TDB = 64;         // dumbbell records per shared-memory tile
constexpr int NA_MAX_CHUNKS = 16;  // j-split chunks at most

// Layout of the static scratch array (bytes, each region 256-byte aligned).
constexpr size_t REC_BYTES = (size_t)DBS_NOALLOC_MAX_S * sizeof(DbF32);
constexpr size_t PART_BYTES = (size_t)NA_MAX_CHUNKS * DBS_NOALLOC_MAX_S * 12 * sizeof(float);
constexpr size_t TICKET_BYTES = ((DBS_NOALLOC_MAX_S + NA_BT - 1) / NA_BT) * sizeof(unsigned);
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t OFF_REC = 0;
constexpr size_t OFF_PART = OFF_REC + align256(REC_BYTES);
constexpr size_t OFF_TICKET = OFF_PART + align256(PART_BYTES);
constexpr size_t OFF_MISC = OFF_TICKET + align256(TICKET_BYTES);  // flags (int) + step (int64)
constexpr size_t SCRATCH_BYTES = OFF_MISC + 256;

// The scratch: one copy per device that loads the library, held until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[MAX_DEVICES] = {};
int g_grid_occ[MAX_DEVICES] = {};  // resident CTAs per SM of the apply kernel
int g_sms[MAX_DEVICES] = {};

const double PI_NA = 3.14159265358979323846;

// One-time set-up per device (that device current): the device address of the
// scratch array and the occupancy of the kernel.
int setup_device(int dev)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_dev_ptr[dev]) return DBS_OK;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return DBS_E_CUDA;
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, eval_kernel<float, DBS_RPY, PHASE_APPLY, NA_BT, NA_TDB>, NA_BT,
            eval_smem_bytes<float>(NA_BT, NA_TDB, NA_MAX_CHUNKS)) != cudaSuccess)
        return DBS_E_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DBS_E_CUDA;
    g_grid_occ[dev] = std::max(1, occ);
    g_sms[dev] = std::max(1, sms);
    g_dev_ptr[dev] = (unsigned char *)ptr;
    return DBS_OK;
}

// Pack positions x and the given forces F into dumbbell records (FP32 pair data).
// Positions are taken relative to the first sphere, a point of the suspension,
// before the FP32 rounding: the pair sum needs only differences, and the
// records keep their relative precision wherever the suspension sits.
__global__ void noalloc_pack_kernel(EvalArgs A, const double *F)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.S) return;
    A.cx = A.x[0];
    A.cy = A.x[1];
    A.cz = A.x[2];
    double xq[6], Fq[6];
    for (int k = 0; k < 6; ++k) {
        xq[k] = A.x[6 * s + k];
        Fq[k] = F[6 * s + k];
    }
    store_rec((DbF32 *)A.pack_out, s, xq, Fq, A);
}

}  // namespace

extern "C" DBS_API int dbs_mobility_apply_noalloc(int64_t S, const double *x_dev,
                                                  const double *F_dev, double a, double mu,
                                                  int32_t mobility, double *v_dev, void *stream)
{
    if (S < 1 || S > DBS_NOALLOC_MAX_S) return DBS_E_ARG;  // beyond the fixed scratch
    if (!x_dev || !F_dev || !v_dev) return DBS_E_ARG;
    if (!(a > 0 && mu > 0 && std::isfinite(a) && std::isfinite(mu))) return DBS_E_ARG;
    if (mobility != DBS_OSEEN && mobility != DBS_RPY) return DBS_E_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return DBS_E_CUDA;
    int rc = setup_device(dev);
    if (rc != DBS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = g_dev_ptr[dev];

    // work split: 32 dumbbells per i-block, C chunks filling whole waves (at most 16)
    const int64_t iblocks = (S + NA_BT - 1) / NA_BT;
    const int64_t gfull = (int64_t)g_sms[dev] * g_grid_occ[dev];
    const int64_t max_chunks = std::max<int64_t>(1, std::min<int64_t>(NA_MAX_CHUNKS, S / 16));
    int64_t C = 1;
    {
        double best = 1e300;
        for (int64_t c = 1; c <= max_chunks; ++c) {
            const int64_t u = iblocks * c;
            best = std::min(best, (double)((u + gfull - 1) / gfull * gfull) / (double)u);
        }
        for (int64_t c = 1; c <= max_chunks; ++c) {
            const int64_t u = iblocks * c;
            if ((double)((u + gfull - 1) / gfull * gfull) / (double)u <= best * 1.01) {
                C = c;
                break;
            }
        }
    }

    EvalArgs A{};
    A.S = S;
    A.N = 2 * S;
    A.x = const_cast<double *>(x_dev);
    A.Fd = const_cast<double *>(F_dev);  // self term reads F through Fd (not written in APPLY)
    A.pack_in = base + OFF_REC;
    A.pack_out = base + OFF_REC;
    A.vout = v_dev;
    A.part = (float *)(base + OFF_PART);
    A.tickets = (unsigned *)(base + OFF_TICKET);
    A.flags = (int *)(base + OFF_MISC);
    A.step = (int64_t *)(base + OFF_MISC + 8);
    A.a = a;
    A.inv6pimua = 1.0 / (6.0 * PI_NA * mu * a);
    A.inv8pimu = 1.0 / (8.0 * PI_NA * mu);
    A.inv8pimu_f = (float)A.inv8pimu;
    A.c2 = (float)(2.0 * a * a / 3.0);
    A.c3 = (float)(-2.0 * a * a);
    A.overlap_r2 = (float)(4.0 * a * a);
    A.chunks = (int)C;
    A.ib0 = 0;
    A.nib = (int)iblocks;
    A.apply_self = 1;

    // the arrival tickets, fault flags and step word start at zero on every call
    if (cudaMemsetAsync(base + OFF_TICKET, 0, OFF_MISC + 16 - OFF_TICKET, st) != cudaSuccess)
        return DBS_E_CUDA;
    noalloc_pack_kernel<<<(int)((S + 127) / 128), 128, 0, st>>>(A, F_dev);
    const int grid = (int)std::min<int64_t>(gfull, iblocks * C);
    const size_t smem = eval_smem_bytes<float>(NA_BT, NA_TDB, (int)C);
    if (mobility == DBS_RPY)
        eval_kernel<float, DBS_RPY, PHASE_APPLY, NA_BT, NA_TDB><<<grid, NA_BT, smem, st>>>(A);
    else
        eval_kernel<float, DBS_OSEEN, PHASE_APPLY, NA_BT, NA_TDB><<<grid, NA_BT, smem, st>>>(A);
    if (cudaGetLastError() != cudaSuccess) return DBS_E_CUDA;
    int flags = 0;
    if (cudaMemcpyAsync(&flags, base + OFF_MISC, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return DBS_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DBS_E_CUDA;
    if (flags & FLAG_OVERLAP) return DBS_E_OVERLAP;
    if (flags & FLAG_NONFINITE) return DBS_E_NONFINITE;
    return DBS_OK;
}
