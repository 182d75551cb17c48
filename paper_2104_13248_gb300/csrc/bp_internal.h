// Internal declarations shared by the libbp translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <string>
#include <vector>

#include "../../include/bp.h"

namespace bp {

// Device error word values (bit flags, OR-ed by kernels).
enum : unsigned {
    DEV_ERR_TIMEOUT = 1u,    // a bounded mbarrier wait ran out
    DEV_ERR_FOOTPRINT = 2u,  // a view's footprint did not fit the staged box
};

// Per (CTA tile, view) geometry record, computed in FP64 from the projection
// matrix and rounded to FP32 once (Section 3.1.2 hoisting: u and w depend
// only on the column (i, j), v is affine in k). Coordinates are relative to
// the integer origin (u_box, v_box) of the staged detector box, so the FP32
// values are small and keep ~1e-5 px accuracy:
//   W(di,dj)     = W0 + Wi*di + Wj*dj                (depth, 1 at isocenter)
//   u - u_box    = (Nu0 + Nui*di + Nuj*dj) / W
//   v - v_box    = (Nv0 + Nvi*di + Nvj*dj + Nvk*dk) / W
// where (di, dj, dk) is the voxel offset from the tile origin.
struct __align__(16) ViewRec {
    float Nu0, Nui, Nuj, W0;
    float Nv0, Nvi, Nvj, Nvk;
    float Wi, Wj;
    int u_box, v_box;
};
static_assert(sizeof(ViewRec) == 48, "ViewRec layout");

// Same for the per-voxel kernel used with general matrices (u and w may
// depend on k as well): u - u_ref = (Nu0 + Nui di + Nuj dj + Nuk dk) / W etc.
struct __align__(16) ViewRecGen {
    float Nu0, Nui, Nuj, Nuk;
    float Nv0, Nvi, Nvj, Nvk;
    float W0, Wi, Wj, Wk;
    int u_ref, v_ref, pad0, pad1;
};
static_assert(sizeof(ViewRecGen) == 64, "ViewRecGen layout");

// Launch plan of the z-column kernels (chosen at create time).
struct Plan {
    int tx, ty, tk;          // CTA tile in voxels (x, y, z); one thread per column
    int bu, bv;              // staged detector box (columns, rows), per dtype below
    int bu16;                // box width for FP16 (multiple of 8)
    int stages;              // pipeline depth (views in flight), <= the requested depth
    int sym_bu, sym_bv;      // mid-plane symmetry kernel: staged box (16-voxel half columns), -1 if off
    int ctas;                // CTAs per SM the TK=32 kernel's register budget targets (2 or 3)
    int fp_wbu;              // forward projector: window width in columns (8 x 4 column patch), -1 if unusable
};

}  // namespace bp

struct bp_ctx {
    int device = 0;
    int n_allocs = 0;           // device allocations made by bp_create (test hook count)
    int n_views = 0, nu = 0, nv = 0, nx = 0, ny = 0, nz = 0;
    bool has_geometry = false;  // created by bp_create (filter, phantom available)
    bool zinv = false;          // every view has P[0][2] = P[2][2] = 0
    bp_geometry g{};
    std::vector<double> angles;
    std::vector<double> P;      // [np][12] FP64 (host copy)
    double *d_P = nullptr;      // [np][12] FP64 (device)
    unsigned *d_err = nullptr;  // device error word
    // ramp filter
    int stages_req = 4;         // requested back-projector pipeline depth (bp_set_pipeline_depth)
    int sym_enable = 1;         // mid-plane symmetry allowed (bp_set_symmetry; used when the matrices have it)
    int fft_n = 0, fft_log2 = 0;
    float *d_H = nullptr;       // [fft_n] real spectrum (times dp, times 1/N), natural order
    float2 *d_tw = nullptr;     // [fft_n] twiddles exp(-2 pi i k / N)
    int fft_quad = 0;           // 1: four-row kernel (tables d_ctH, d_cttw), 0: two-row kernel (d_H, d_tw)
    void *d_ctH = nullptr;      // [16][fft_n / 16] float2 (H sdd, H sdd) at the fused step's positions
    void *d_cttw = nullptr;     // [ct_twiddle_count] float4 (cos, cos, sin, sin) per pass and (k, o)
    float *d_phcoef = nullptr;  // [np][256][20] phantom coefficients (input generation)
    // launch plan
    bp::Plan plan{};
    int sm_count = 0;
    unsigned long long timeout_ns = 2000000000ull;  // bounded waits in kernels
    int test_drop_view = -1;    // test hook: producer skips this view's load (-1: off)
    std::string err;
};

namespace bp {

// Error helpers (bp_api.cu).
bp_status fail(bp_ctx *ctx, bp_status st, const std::string &msg);
bp_status cuda_fail(bp_ctx *ctx, cudaError_t e, const char *what);

// Kernel launchers (one per translation unit). They validate nothing the
// API layer already checked; they return BP_ERR_CUDA on a launch failure.
// Slices [z0, z0 + nzs) and, with mirror, [nz - z0 - nzs, nz - z0).
bp_status launch_backproject(bp_ctx *ctx, const void *proj, bp_dtype t, int view0, int nviews,
                             long long batch_stride, float *vol, int batch, float scale,
                             int accumulate, cudaStream_t st, int z0, int nzs, int mirror);
bp_status launch_forward(bp_ctx *ctx, const float *vol, float *proj, int batch, float scale,
                         cudaStream_t st);
// Dynamic shared memory of the forward projector for windows wc columns wide.
int fp_smem_bytes(int wc);
int fp_window_width(int need);   // smallest window width the forward projector is built for, or -1
bp_status launch_filter(bp_ctx *ctx, const float *proj, void *out, bp_dtype out_t,
                        long long n_views_total, cudaStream_t st);
bp_status launch_phantom(bp_ctx *ctx, const double *d_ell, int n_ell, float *proj,
                         cudaStream_t st);

// Footprint bound used by the plan: the largest staged box (columns, rows)
// any tile needs in any view, from the FP64 matrices (bp_api.cu).
void max_footprint(const bp_ctx *ctx, int tx, int ty, int tk, int align, int *bu, int *bv);

}  // namespace bp
