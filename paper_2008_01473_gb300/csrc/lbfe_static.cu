// lb_fields_static: the field-export and reduction pass of lb_moments /
// lb_reductions for callers that cannot allocate device memory. Its scratch
// lives in a file-scope device array of fixed size instead of the caller's
// workspace; see include/lbfe.h for the contract.
#include <cmath>
#include <mutex>

#include "../../include/lbfe.h"
#include "aux_kernels.cuh"

using namespace lbfe;

namespace {

constexpr int64_t kMaxNodes = LB_STATIC_MAX_NODES;
constexpr int kMaxSide = LB_STATIC_MAX_SIDE;
// partials of velocity_kernel: at most ceil(nx / 256) * ny <= nodes / 256 + ny
constexpr int64_t kMaxParts = kMaxNodes / 256 + kMaxSide;
constexpr size_t kFieldBytes = kMaxNodes * sizeof(double);
constexpr size_t kScratchBytes = 4 * kFieldBytes + kMaxParts * sizeof(Partial);

constexpr int kMaxDevices = 256;
template <typename T>
DevCase<T> make_case(const lb_case& c, double rho_ref)
{
    DevCase<T> d{};
    d.nx = c.nx;
    d.ny = c.ny;
    d.pitch = pitch_of(c.nx);
    d.off = 0;
    d.plane = (int64_t)c.ny * d.pitch;
    d.RT = (T)(c.R * c.T);
    d.a = (T)c.a;
    d.b = (T)c.b;
    d.kappa = (T)c.kappa;
    d.c0 = (T)c.pm_c0;
    d.rho_ref = (T)rho_ref;
    return d;
}

bool valid_case(const lb_case& c)
{
    if (c.nx < 3 || c.ny < 3) return false;
    if (c.scheme != LB_STANDARD && c.scheme != LB_IMPROVED && c.scheme != LB_IMPROVED_SMOOTH) return false;
    if (c.walls) return false;  // periodic lattices only
    if (c.eos != LB_VDW && c.eos != LB_CS) return false;
    const double v[] = {c.a, c.b, c.R, c.T, c.kappa, c.pm_c0};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return c.a > 0 && c.b > 0 && c.R > 0 && c.T > 0 && c.kappa > 0;
}

}  // namespace

// Scratch of lb_fields_static: shared by every call on a device and held by
// every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in, not a device address).
cudaError_t scratch_ptr(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}
}  // namespace

// The pass of lb_moments / lb_reductions in the storage precision T of the
// populations (per-node arithmetic in T, sums in FP64), on the static scratch.
template <typename T>
void fields_static(const lb_case& c, double rho_ref, const T* d_pops, unsigned char* p, Partial* parts,
                   double* d_rho, double* d_ux, double* d_uy, double* d_mu, dim3 grd, dim3 blk, cudaStream_t st)
{
    T* s0 = reinterpret_cast<T*>(p);
    T* s1 = reinterpret_cast<T*>(p + kFieldBytes);
    T* s2 = reinterpret_cast<T*>(p + 2 * kFieldBytes);
    T* s3 = reinterpret_cast<T*>(p + 3 * kFieldBytes);
    const DevCase<T> ct = make_case<T>(c, rho_ref);
    pull_moments_kernel<T, T><<<grd, blk, 0, st>>>(ct, d_pops, s0, s1, s2);
    if (c.eos == LB_VDW)
        mu_field_kernel<T, 0><<<grd, blk, 0, st>>>(ct, s0, s3);
    else
        mu_field_kernel<T, 1><<<grd, blk, 0, st>>>(ct, s0, s3);
    if (improved_scheme(c.scheme))  // the exported fields do not involve Eq. 29
        velocity_kernel<1, T><<<grd, blk, 0, st>>>(ct, s0, s1, s2, s3, nullptr, nullptr, nullptr, d_rho, d_ux, d_uy,
                                                   d_mu, parts);
    else
        velocity_kernel<0, T><<<grd, blk, 0, st>>>(ct, s0, s1, s2, s3, nullptr, nullptr, nullptr, d_rho, d_ux, d_uy,
                                                   d_mu, parts);
}

extern "C" lb_status lb_fields_static(const lb_case* c, int32_t precision, const void* d_pops,
                                      double rho_ref, double* d_rho, double* d_ux, double* d_uy,
                                      double* d_mu, double* d_red, void* cuda_stream)
{
    if (!c || !d_pops || !d_red || !valid_case(*c)) return LB_E_INVALID;
    if (precision != LB_FP32 && precision != LB_FP64) return LB_E_INVALID;
    if (!std::isfinite(rho_ref) || rho_ref < 0) return LB_E_INVALID;
    if (c->nx > kMaxSide || c->ny > kMaxSide || (int64_t)c->nx * c->ny > kMaxNodes) return LB_E_INVALID;
    // an error left pending by earlier work is not this call's to report or
    // to clear: leave it in place and enqueue nothing
    if (cudaPeekAtLastError() != cudaSuccess) return LB_E_CUDA;
    void* base = nullptr;
    if (scratch_ptr(&base) != cudaSuccess) return LB_E_CUDA;
    unsigned char* p = static_cast<unsigned char*>(base);
    Partial* parts = reinterpret_cast<Partial*>(p + 4 * kFieldBytes);
    // Every scratch value read below is written earlier in the same call
    // (all nodes of the four fields, all partials of the grid), so nothing
    // needs clearing between calls.
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const dim3 blk(256), grd = field_grid(c->nx, c->ny);
    if (precision == LB_FP32)
        fields_static<float>(*c, rho_ref, (const float*)d_pops, p, parts, d_rho, d_ux, d_uy, d_mu, grd, blk, st);
    else
        fields_static<double>(*c, 0.0, (const double*)d_pops, p, parts, d_rho, d_ux, d_uy, d_mu, grd, blk, st);
    finalize_kernel<<<1, 256, 0, st>>>(parts, (int64_t)grd.x * grd.y, 0.0, d_red);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_E_CUDA;
}
