// Read-only view of a problem's device data for entry points that live
// outside api.cu. Building the view allocates nothing.
#pragma once

#include "common.cuh"
#include "conv.cuh"

namespace bae {

struct ProblemView {
    int device = 0;
    int N = 0;
    long long n_gm = 0;
    long long n_unk = 0;              // unknowns: n_gm, or n_gm + |gamma+| (direct formulation)
    cudaStream_t stream = nullptr;
    SrcRecipe rec;
    const double* ghat64 = nullptr;   // octant spectrum, 1/(2N)^3 folded in
    const float* ghat32 = nullptr;
    const double2* tw64 = nullptr;    // exp(-2 pi i m / 2N); null if not built yet
    const float2* tw32 = nullptr;
};

// Fills `out` from a problem handle (no device work, no allocation).
bool problem_view(const bae_problem* P, ProblemView& out);

// Makes dst use src's LGF spectrum cache (contexts of one server share it).
void ctx_share_cache(bae_ctx* dst, const bae_ctx* src);
// marks a context whose GPU runs other contexts' kernels at the same time
// (a server slot): it launches no cooperative kernel
void ctx_set_shared_gpu(bae_ctx* c);

}  // namespace bae
