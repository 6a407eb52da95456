// Point sets, closure and source stencil of a problem (Section 2.1, 3.2).
#pragma once

#include "common.cuh"
#include "conv.cuh"

namespace bae {

// Owning device arrays describing one classified grid.
struct Geometry {
    int N = 0;
    double h = 0.0;
    double origin[3] = {0, 0, 0};
    int layer = BAE_LAYER_DOUBLE;
    cudaStream_t stream = nullptr;  // stream that owns the allocations
    long long n_gm = 0, n_gp = 0, n_mp = 0, n_src = 0, n_terms = 0;
    long long n_unk = 0;          // unknowns: n_gm, or n_gm + n_gp (direct formulation: u on gamma- then gamma+)
    uint8_t* flags = nullptr;     // N^3: bit0 M+, bit1 gamma-, bit2 gamma+, bit3 D-node, bits4-6 |D_n|
    int* gm = nullptr;            // gamma- linear indices, lexicographic
    int* gp = nullptr;            // gamma+ linear indices, lexicographic
    int* node_of = nullptr;       // N^3: unknown number of a gamma node (gamma-: its gm index, gamma+: n_gm + gp index; set there only)
    int* partner_u = nullptr;     // direct formulation: unknown number of each gamma- node's partner
    int* partner = nullptr;       // closure partner per gamma- node
    double* t = nullptr;          // closure weight per gamma- node
    double* xstar = nullptr;      // boundary points, 3 per gamma- node
    int* line_off = nullptr;      // source recipe (see SrcRecipe)
    int* src_lin = nullptr;
    int* term_off = nullptr;
    int* term_idx = nullptr;
    double* term_coef = nullptr;
    float* term_coef32 = nullptr;  // the coefficients rounded to float32 (small integers and 6 + s)
    // x-planes [plane_lo, plane_hi) contain every source and every node the
    // gather and the reconstruction read
    int plane_lo = 0, plane_hi = 0;
    // the same range along each axis (0: x, 1: y, 2: z)
    int ext_lo[3] = {0, 0, 0}, ext_hi[3] = {0, 0, 0};

    // Swapped view of the pruned applies: the convolution skips the zero
    // planes of its first axis only, so it runs on the grid with axis 0
    // swapped with the axis of fewest planes (cv_swap, see swap_axes; 0: no
    // swap, where x is already the narrowest, for the direct formulation and
    // when BAE_CONV_AXIS=x). cv_lo/cv_hi is the plane range along that axis;
    // the recipe, the flags and the gathered indices below are the
    // geometry's in the swapped layout (null when cv_swap == 0).
    int cv_swap = 0;
    int cv_lo = 0, cv_hi = 0;
    uint8_t* cv_flags = nullptr;
    int* cv_gm = nullptr;
    int* cv_partner = nullptr;
    int* cv_line_off = nullptr;
    int* cv_src_lin = nullptr;
    int* cv_term_off = nullptr;
    int* cv_term_idx = nullptr;
    double* cv_term_coef = nullptr;
    float* cv_term_coef32 = nullptr;

    SrcRecipe recipe() const {
        SrcRecipe r;
        r.line_off = line_off;
        r.src_lin = src_lin;
        r.term_off = term_off;
        r.term_idx = term_idx;
        r.term_coef = term_coef;
        r.term_coef32 = term_coef32;
        r.wide = layer == BAE_LAYER_DIRECT;
        return r;
    }
    // the recipe of the swapped view (the plain one when cv_swap == 0)
    SrcRecipe cv_recipe() const {
        if (!cv_swap) return recipe();
        SrcRecipe r;
        r.line_off = cv_line_off;
        r.src_lin = cv_src_lin;
        r.term_off = cv_term_off;
        r.term_idx = cv_term_idx;
        r.term_coef = cv_term_coef;
        r.term_coef32 = cv_term_coef32;
        r.wide = layer == BAE_LAYER_DIRECT;
        return r;
    }
    void release();
};

// Classifies phi (device, N^3 float64), builds the closure and the source
// recipe. Throws Error(BAE_ERR_GEOMETRY) when gamma- is empty or when M+ or
// gamma- reaches the box faces, Error(BAE_ERR_INVALID_ARG) on non-finite phi.
// s = kappa^2 h^2 (the direct formulation's source stencil uses 6 + s).
void build_geometry(const double* phi, int N, double h, const double origin[3], int layer, double s,
                    Geometry& g, cudaStream_t st);

}  // namespace bae
