// Allocation-free Morton ordering of a particle set.
//
// Some callers cannot let a library allocate device memory: simulation
// codes that hand out every byte of the GPU from their own pool or from a
// budget fixed at start-up, and codes that must not stall mid-step, since
// cudaMalloc / cudaFree synchronise the whole device and hold up the
// caller's other streams.  For them this file offers one entry point that
// orders particles exactly as start_build_trees does (root frame, 63-bit
// Morton keys, stable radix sort by key then input index) but takes all of
// its scratch from a fixed array compiled into the library.
//
// The scratch is a file-scope __device__ array sized for at most
// kNoAllocMaxN particles (about 20.5 MB).  Every GPU that loads this part of
// the library keeps that array until the process exits.  All calls share
// it, so calls whose work overlaps on the GPU (two streams, or two host
// threads) race and corrupt each other's results; serialise them.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace st {

// Kernels of the regular path (scan_sort.cu), reused unchanged with
// pointers into the fixed scratch.
__global__ void k_bbox_init(int *mm);
__global__ void k_bbox(const float *pos, long long n, int *mm, unsigned long long *bad);
__global__ void __launch_bounds__(256) k_rs_hist(const u64 *keys, long long n, int shift,
                                                 u32 *hist, int nblocks);
__global__ void __launch_bounds__(256) k_rs_scatter(const u64 *kin, const u32 *vin, u64 *kout,
                                                    u32 *vout, long long n, int shift,
                                                    const u32 *offs, int nblocks);

namespace {

constexpr long long kNoAllocMaxN = 1LL << 20;
constexpr int kTile = 4096;                               // items per sort block
constexpr int kMaxBlocks = (int)(kNoAllocMaxN / kTile);   // 256
constexpr size_t kHeader = 256;
constexpr size_t kKeysA = kHeader;
constexpr size_t kKeysB = kKeysA + (size_t)kNoAllocMaxN * 8;
constexpr size_t kValsB = kKeysB + (size_t)kNoAllocMaxN * 8;
constexpr size_t kHist = kValsB + (size_t)kNoAllocMaxN * 4;
constexpr size_t kOffs = kHist + (size_t)256 * kMaxBlocks * 4;
constexpr size_t kScratchBytes = kOffs + (size_t)256 * kMaxBlocks * 4;

// Header layout: int mm[6] at 0, u64 bad at 32, double frame[5] at 64.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device; looked up
// once per device (the host-side name of the array is only a stand-in).
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return START_ECUDA;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return START_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return START_OK;
}

// True when p is device (or managed) memory of the current device.
bool on_device(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

__device__ __forceinline__ float ord_to_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Root frame from the reduced bounding box, with the same FP64 operations
// as the host-side frame of start_build_trees: lower corner = minima,
// side = largest extent (1 if zero), scale = 2^21 / side.
__global__ void k_frame_dev(const int *mm, double *frame, double *frame_out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo[3], side = 0.0;
    for (int a = 0; a < 3; ++a) {
        lo[a] = (double)ord_to_float(mm[a]);
        double e = __dsub_rn((double)ord_to_float(mm[3 + a]), lo[a]);
        if (e > side) side = e;
    }
    if (!(side > 0.0)) side = 1.0;
    for (int a = 0; a < 3; ++a) frame[a] = lo[a];
    frame[3] = side;
    frame[4] = __ddiv_rn(2097152.0, side);
    if (frame_out)
        for (int a = 0; a < 4; ++a) frame_out[a] = frame[a];
}

__device__ __forceinline__ u64 spread3_na(u64 v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Morton keys with the frame read from device memory (no host round trip).
__global__ void k_morton_dev(const float *pos, long long n, const double *frame, u64 *keys,
                             u64 *keys_copy, u32 *idx)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double scale = frame[4];
    u64 q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double t = floor(__dmul_rn(__dsub_rn((double)pos[(long long)a * n + i], frame[a]), scale));
        t = fmin(fmax(t, 0.0), 2097151.0);
        q[a] = (u64)t;
    }
    u64 k = (spread3_na(q[0]) << 2) | (spread3_na(q[1]) << 1) | spread3_na(q[2]);
    keys[i] = k;
    keys_copy[i] = k;
    idx[i] = (u32)i;
}

// Exclusive scan of the 256 x nblocks digit histogram in one block.
__global__ void __launch_bounds__(1024) k_scan_hist(const u32 *in, u32 *out, int m)
{
    __shared__ u32 part[1024];
    int t = threadIdx.x;
    int per = (m + 1023) / 1024;
    int b = t * per, e = min(m, b + per);
    u32 s = 0;
    for (int i = b; i < e; ++i) s += in[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        u32 v = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    u32 run = t ? part[t - 1] : 0u;
    for (int i = b; i < e; ++i) {
        u32 v = in[i];
        out[i] = run;
        run += v;
    }
}

}  // namespace
}  // namespace st

using namespace st;

extern "C" int start_morton_order_noalloc(const float *pos, long long n, unsigned long long *keys_out,
                                          unsigned *perm_out, double *frame_out, void *stream)
{
    if (n < 0) return START_EINVAL;
    if (n > kNoAllocMaxN) return START_ERANGE;
    if (n == 0) return START_OK;
    if (!pos || !keys_out || !perm_out) return START_EINVAL;
    // kernels read and write these directly: host memory is refused
    if (!on_device(pos) || !on_device(keys_out) || !on_device(perm_out) ||
        (frame_out && !on_device(frame_out)))
        return START_EINVAL;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != START_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *sc = static_cast<unsigned char *>(base);
    int *mm = reinterpret_cast<int *>(sc);
    unsigned long long *bad = reinterpret_cast<unsigned long long *>(sc + 32);
    double *frame = reinterpret_cast<double *>(sc + 64);
    u64 *ka = reinterpret_cast<u64 *>(sc + kKeysA);
    u64 *kb = reinterpret_cast<u64 *>(sc + kKeysB);
    u32 *vb = reinterpret_cast<u32 *>(sc + kValsB);
    u32 *hist = reinterpret_cast<u32 *>(sc + kHist);
    u32 *offs = reinterpret_cast<u32 *>(sc + kOffs);
    int nblocks = (int)((n + kTile - 1) / kTile);

    // the array keeps the previous call's contents: reset the counter
    if (cudaMemsetAsync(bad, 0, sizeof(*bad), s) != cudaSuccess) return START_ECUDA;
    k_bbox_init<<<1, 32, 0, s>>>(mm);
    k_bbox<<<grid_for(n, 256, 1024), 256, 0, s>>>(pos, n, mm, bad);
    k_frame_dev<<<1, 1, 0, s>>>(mm, frame, frame_out);
    k_morton_dev<<<grid_for(n, 256), 256, 0, s>>>(pos, n, frame, ka, reinterpret_cast<u64 *>(keys_out),
                                                  perm_out);
    u64 *k0 = ka, *k1 = kb;
    u32 *v0 = perm_out, *v1 = vb;
    for (int pass = 0; pass < 8; ++pass) {
        k_rs_hist<<<nblocks, 256, 0, s>>>(k0, n, 8 * pass, hist, nblocks);
        k_scan_hist<<<1, 1024, 0, s>>>(hist, offs, 256 * nblocks);
        k_rs_scatter<<<nblocks, 256, 0, s>>>(k0, v0, k1, v1, n, 8 * pass, offs, nblocks);
        u64 *tk = k0; k0 = k1; k1 = tk;
        u32 *tv = v0; v0 = v1; v1 = tv;
    }
    // eight passes: the sorted order is back in perm_out
    if (cudaGetLastError() != cudaSuccess) return START_ECUDA;
    unsigned long long nbad = 0;
    if (cudaMemcpyAsync(&nbad, bad, sizeof(nbad), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return START_ECUDA;
    }
    return nbad ? START_EINVAL : START_OK;
}
