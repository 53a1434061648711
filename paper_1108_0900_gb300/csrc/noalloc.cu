// Allocation-free variant of the pairing-block half of the S product.
//
// Some callers cannot call cudaMalloc: code that runs inside a fixed memory
// budget owned by a pool allocator (a framework's caching allocator can hold
// every free byte, so a fresh cudaMalloc fails), and latency-critical loops,
// where cudaMalloc / cudaFree synchronise the device.  For them this file
// offers sr_pairing_product_noalloc: the caller passes every input and output,
// and the only scratch - one partial image of the pairing block per CTA - lives
// in a fixed file-scope device array.
//
// The kernel is a variant of the generic streaming pass (sr.cu, k_sr_main with
// FP32 storage and accumulation): warp per sample, t_s = W_s . v over the
// pairing block, then sum_s t_s W_s into a shared-memory image per CTA, which
// is written to the static scratch and reduced in FP64 by a second kernel.
#include <mutex>
#include <string>

#include "common.cuh"
#include "vmcsr.h"

namespace vmc {

constexpr int kNoallocMaxCtas = 128;
constexpr int kNoallocMaxNpf = 128 * 127 / 2;  // pairing block of 128 spin orbitals

// Fixed scratch shared by every call on a device (4.2 MB): CTA images of the
// pairing block.  Held by each GPU that loads the library until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[kNoallocMaxCtas * kNoallocMaxNpf];

__global__ void __launch_bounds__(512) k_pairing_product_static(int64_t n_s, int M, int nu, int nd,
                                                                const uint8_t* occ, int64_t occ_stride,
                                                                const float* pf, int64_t pf_stride,
                                                                const float* v, float* t_out, float* scratch) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int npf = M * (M - 1) / 2, N = nu + nd;
    const int P = nu * (nu - 1) / 2 + nd * (nd - 1) / 2 + nu * nd;
    float* acc = (float*)smem;
    float* vpf = acc + npf;
    uint16_t* pairs = (uint16_t*)(vpf + npf);
    uint8_t* occw = (uint8_t*)(pairs + ((P + 7) & ~7));
    for (int i = threadIdx.x; i < npf; i += blockDim.x) {
        acc[i] = 0.f;
        vpf[i] = v[i];
    }
    // pair decode table in the documented block order: up-up triangle,
    // down-down triangle, up-down rectangle, each row-major
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        int a, b, r = e;
        const int puu = nu * (nu - 1) / 2, pdd = nd * (nd - 1) / 2;
        if (r < puu) {
            a = 0;
            while (r >= nu - 1 - a) { r -= nu - 1 - a; ++a; }
            b = a + 1 + r;
        } else if (r < puu + pdd) {
            r -= puu;
            a = 0;
            while (r >= nd - 1 - a) { r -= nd - 1 - a; ++a; }
            b = nu + a + 1 + r;
            a += nu;
        } else {
            r -= puu + pdd;
            a = r / nd;
            b = nu + r % nd;
        }
        pairs[e] = (uint16_t)(a | (b << 8));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint8_t* my = occw + wid * 64;
    const int ns = M >> 1;
    for (int64_t s = (int64_t)blockIdx.x * nw + wid; s < n_s; s += (int64_t)gridDim.x * nw) {
        // the occupation must be a configuration of the sector: strictly
        // ascending, n_up orbitals below n_sites, n_dn from n_sites to M - 1;
        // otherwise some pairing index would fall outside the images, so the
        // sample gets t_s = NaN and adds nothing
        bool bad = false;
        for (int i = lane; i < N; i += 32) {
            const int o = occ[s * occ_stride + i];
            my[i] = (uint8_t)o;
            const bool spin_ok = i < nu ? o < ns : (o >= ns && o < M);
            const bool asc = i == 0 || o > (int)occ[s * occ_stride + i - 1];
            bad = bad || !spin_ok || !asc;
        }
        if (__any_sync(VMC_FULL_MASK, bad)) {
            if (lane == 0) t_out[s] = __int_as_float(0x7fc00000);
            __syncwarp();
            continue;
        }
        __syncwarp();
        const float* W = pf + s * pf_stride;
        float t = 0.f;
        for (int e = lane; e < P; e += 32) {
            const uint16_t pt = pairs[e];
            const int p = my[pt & 255], q = my[pt >> 8];
            t += W[e] * vpf[(int)pf_row_base(M, p) + q];
        }
        t = warp_sum(t);
        if (lane == 0) t_out[s] = t;
        for (int e = lane; e < P; e += 32) {
            const uint16_t pt = pairs[e];
            const int p = my[pt & 255], q = my[pt >> 8];
            atomicAdd(&acc[(int)pf_row_base(M, p) + q], t * W[e]);
        }
        __syncwarp();
    }
    __syncthreads();
    float* dst = scratch + (size_t)blockIdx.x * npf;
    for (int i = threadIdx.x; i < npf; i += blockDim.x) dst[i] = acc[i];
}

__global__ void k_pairing_reduce_static(const float* scratch, int nblk, int npf, double* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npf; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += (double)scratch[(size_t)b * npf + i];
        out[i] = s;
    }
}

}  // namespace vmc

using namespace vmc;

namespace vmc {
void set_error_detail(const std::string& s);  // api.cu: text for vmc_last_error_detail
}

namespace {
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[64] = {};     // device address of the scratch, per device
int g_noalloc_sms[64] = {};
}  // namespace

extern "C" int sr_pairing_product_noalloc(int64_t n_s, int n_sites, int n_up, int n_dn, const uint8_t* occ,
                                          int64_t occ_stride, const float* pf, int64_t pf_stride, const float* v,
                                          float* t, double* out, void* stream) {
    if (n_sites > 64) {
        set_error_detail("sr_pairing_product_noalloc: more than 64 sites exceeds the fixed scratch "
                         "(at most 8128 pairing amplitudes)");
        return VMC_ERR_INVALID_ARG;
    }
    const int M = 2 * n_sites, N = n_up + n_dn;
    const int npf = M * (M - 1) / 2;
    const int P = n_up * (n_up - 1) / 2 + n_dn * (n_dn - 1) / 2 + n_up * n_dn;
    if (n_sites < 1 || n_up < 0 || n_dn < 0 || n_up > n_sites || n_dn > n_sites || N < 2 || N > 64 ||
        n_s < 0 || (n_s > 0 && (!occ || !pf || !t)) || !v || !out || occ_stride < N || pf_stride < P) {
        set_error_detail("sr_pairing_product_noalloc: invalid sizes, strides or pointers");
        return VMC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return VMC_ERR_CUDA;
    float* scratch;
    int sms;
    {
        // once per device, with that device current: the host-side symbol is
        // only a stand-in, the kernel needs the device address
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                set_error_detail(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return VMC_ERR_CUDA;
            }
            int n = 0;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return VMC_ERR_CUDA;
            g_noalloc_sms[dev] = n;
            g_noalloc_ptr[dev] = (float*)p;
        }
        scratch = g_noalloc_ptr[dev];
        sms = g_noalloc_sms[dev];
    }
    if (n_s == 0) {
        if (cudaMemsetAsync(out, 0, sizeof(double) * npf, st) != cudaSuccess) return VMC_ERR_CUDA;
        return VMC_OK;
    }
    const size_t smem = (size_t)npf * 8 + (size_t)((P + 7) & ~7) * 2 + 16 * 64;
    if (cudaFuncSetAttribute(k_pairing_product_static, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return VMC_ERR_CUDA;
    int grid = sms < kNoallocMaxCtas ? sms : kNoallocMaxCtas;
    const int64_t need = (n_s + 15) / 16;
    if (need < grid) grid = (int)need;
    k_pairing_product_static<<<grid, 512, smem, st>>>(n_s, M, n_up, n_dn, occ, occ_stride, pf, pf_stride, v, t,
                                                      scratch);
    k_pairing_reduce_static<<<(npf + 255) / 256, 256, 0, st>>>(scratch, grid, npf, out);
    if (cudaGetLastError() != cudaSuccess) return VMC_ERR_CUDA;
    return VMC_OK;
}
