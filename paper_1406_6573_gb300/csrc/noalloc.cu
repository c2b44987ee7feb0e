// Fixed-order A-gradient that allocates nothing (a library utility; the
// paper has no counterpart).  The A-gradient lambda^T d r_c / d A (the
// volume integral -(1/(n A)) int mu D(lambda) : D(u), Eq. 2.3 differentiated
// in A) is computed by the element kernel in MODE_GRAD_A_PARTIAL, which
// writes one partial sum per warp into a file-scope device scratch array;
// one block then adds the partials in a fixed order.  The scratch is a
// static __device__ array: its address is resolved once per device with
// cudaGetSymbolAddress and cached; no call allocates device memory.
#include <mutex>

#include <cuda_runtime.h>

#include "handles.h"
#include "kernels.h"

namespace stokes {
namespace {

constexpr int RED_T = 256;

static __device__ __align__(256) double g_grad_a_partials[STOKES_GRAD_A_MAX_PARTIALS];

// out[0] = scale * sum_{w < n} part[w]: thread t adds part[t], part[t + RED_T],
// ... in index order, then a fixed binary tree over the threads.
__global__ void __launch_bounds__(RED_T) fixed_order_sum(const double* __restrict__ part, int64_t n,
                                                         double scale, double* __restrict__ out) {
    __shared__ double red[RED_T];
    double s = 0.0;
    for (int64_t w = threadIdx.x; w < n; w += RED_T) s += part[w];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = RED_T / 2; h > 0; h >>= 1) {
        if (int(threadIdx.x) < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = scale * red[0];
}

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[MAX_DEVICES] = {};

// device address of the scratch on `dev` (first use on a device resolves it)
cudaError_t scratch_on(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_grad_a_partials);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace stokes

using namespace stokes;

extern "C" int stokes_param_grad_A_fixed_order(const stokes_mesh* mesh, const stokes_params* params,
                                               const double* up, const double* lambda, double* g_A,
                                               void* stream) {
    int rc = check_common(mesh, STOKES_F64);
    if (rc) return rc;
    if ((rc = check_params(mesh, params))) return rc;
    if (!up || !lambda || !g_A) return fail(STOKES_E_INVAL, "up, lambda and g_A must be non-NULL device pointers");
    if (mesh->device < 0 || mesh->device >= MAX_DEVICES) return fail(STOKES_E_INVAL, "device ordinal out of range");
    const int64_t nparts = grad_a_partials(mesh->h.k, mesh->h.E);
    if (nparts > STOKES_GRAD_A_MAX_PARTIALS)
        return fail(STOKES_E_INVAL, "mesh needs more A-gradient partial sums than the fixed scratch holds "
                                    "(STOKES_GRAD_A_MAX_PARTIALS)");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* part = nullptr;
    cudaError_t ce = scratch_on(mesh->device, &part);
    if (ce != cudaSuccess) return cuda_fail(ce, "resolving the scratch address");
    if (nparts == 0) {
        ce = cudaMemsetAsync(g_A, 0, sizeof(double), s);
        return ce == cudaSuccess ? STOKES_OK : cuda_fail(ce, "clearing g_A");
    }
    ElemArgs a = elem_args(mesh, params);
    a.ud = up; a.lam = lambda; a.gA_part = part;
    int e = launch_elem(mesh->h.k, MODE_GRAD_A_PARTIAL, STOKES_F64, STOKES_F64, false, a, s);
    if (e) return cuda_fail(cudaError_t(e), "A gradient kernel launch");
    fixed_order_sum<<<1, RED_T, 0, s>>>(part, nparts, -1.0 / (params->n * params->A), g_A);
    ce = cudaGetLastError();
    return ce == cudaSuccess ? STOKES_OK : cuda_fail(ce, "fixed-order sum launch");
}
