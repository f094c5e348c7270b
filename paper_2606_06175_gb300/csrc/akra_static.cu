// akra_static.cu -- spin-2 synthesis that allocates no device memory.
//
// akra_synth_spin2 keeps its phase array Φ in a plan workspace that it grows with
// cudaMalloc on first use (or when R grows).  Some callers cannot allocate at the point
// where they need a synthesis: code running under a device-memory budget or inside a
// memory pool that must not grow, a process where another component (a framework's caching
// allocator, say) has already reserved the device memory, and latency-critical loops where
// a cudaMalloc, with its implicit device synchronisation, is not acceptable.  This entry
// point runs the same two kernels (Legendre synthesis, ring FFT) but puts Φ in a fixed
// file-scope device array instead, so a call allocates nothing.
#include <mutex>

#include "akra_internal.cuh"

namespace akra {

// 32 MiB of scratch for Φ [R][nring][2 lmax + 1] complex.  Every GPU that loads the library
// holds this array until the process exits.
constexpr size_t kStaticScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_phi_scratch[kStaticScratchBytes];

// device address of g_phi_scratch, looked up once per device (the host-side symbol is only
// a stand-in and must never be passed to a kernel)
static std::mutex g_scratch_mu;
static std::map<int, void *> g_scratch_addr;

static akra_status scratch_address(void **out)
{
    int dev = -1;
    AKRA_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    auto it = g_scratch_addr.find(dev);
    if (it != g_scratch_addr.end()) {
        *out = it->second;
        return AKRA_OK;
    }
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_phi_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
        set_error("akra_synth_spin2_static: cudaGetSymbolAddress failed on device %d: %s", dev,
                  cudaGetErrorString(e));
        return AKRA_ECUDA;
    }
    g_scratch_addr[dev] = ptr;
    *out = ptr;
    return AKRA_OK;
}

template <typename T> struct PrecIdxStatic;
template <> struct PrecIdxStatic<float> { static constexpr akra_prec prec = AKRA_F32; };
template <> struct PrecIdxStatic<double> { static constexpr akra_prec prec = AKRA_F64; };

template <typename T>
static akra_status synth_static(akra_plan p, const void *alm, void *map, int R, cudaStream_t st)
{
    const size_t need = (size_t)R * p->nring * (2 * (size_t)p->lmax + 1) * sizeof(cx_t<T>);
    if (need > kStaticScratchBytes) {
        set_error("akra_synth_spin2_static: R * (4 nside - 1) * (2 lmax + 1) complex values need "
                  "%zu bytes, more than the %zu-byte static scratch (use akra_synth_spin2)",
                  need, kStaticScratchBytes);
        return AKRA_EINVAL;
    }
    void *phi = nullptr;
    AKRA_TRY(scratch_address(&phi));
    // every Φ entry the ring FFT reads is written first by the Legendre kernel of this call
    // (all m of all rings), so nothing needs clearing between calls
    // the CUDA-core synthesis: the tensor-core one stages its operand in a plan workspace
    LegShape s = leg_shape(p, PrecIdxStatic<T>::prec, R);
    s.TC = 0;
    AKRA_TRY(legendre_synth<T>(p, s, LegMode::Synth, alm, phi, R, p->d_all_units, p->nunit, st));
    return ring_fft<T>(p, FftMode::Synth, phi, nullptr, map, false, R, p->d_all_rings, p->nring, st);
}

}  // namespace akra

using namespace akra;

extern "C" akra_status akra_synth_spin2_static(akra_plan p, akra_prec prec, const void *d_alm,
                                               void *d_map, int R, void *stream)
{
    AKRA_TRY(reject_flat(p, "akra_synth_spin2_static"));
    if (!p || !d_alm || !d_map) {
        set_error("akra_synth_spin2_static: NULL plan or array");
        return AKRA_EINVAL;
    }
    if (prec != AKRA_F64 && prec != AKRA_F32) {
        set_error("akra_synth_spin2_static: precision must be AKRA_F64 or AKRA_F32");
        return AKRA_EINVAL;
    }
    if (R < 1 || R > 65535) {
        set_error("akra_synth_spin2_static: R = %d outside [1, 65535]", R);
        return AKRA_EINVAL;
    }
    // the plan's tables live on the device it was created on; the scratch looked up below is
    // the current device's, so the two must agree
    int dev = -1;
    AKRA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != p->device) {
        set_error("akra_synth_spin2_static: the current device is %d but the plan was created on "
                  "device %d; make the plan's device current first", dev, p->device);
        return AKRA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return prec == AKRA_F64 ? synth_static<double>(p, d_alm, d_map, R, st)
                            : synth_static<float>(p, d_alm, d_map, R, st);
}
