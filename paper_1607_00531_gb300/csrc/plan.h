// plan.h -- host-side plan of one volume: validated grid, kernel launch
// shapes, and the carving of the caller's workspace.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <memory>
#include <vector>

#include "../../include/sac.h"
#include "sac_dev.cuh"
#include "sac_launch.h"

namespace sac {

struct Geometry {
    int nd, pe;
    int M[3], F[3];
    int ax1, ax2;
    long long nf, nc;
    int n_outer, mpe, n_inner;
    double h[3], hd, hpe;
};

// validate a grid; returns SAC_OK or SAC_EINVAL
int make_geometry(const sac_grid* g, Geometry* out);
int check_params(const sac_params* p);

// DCT-II matrix (orthonormal) and the eigenvalues of the Neumann difference
// operator it diagonalises (Sec. 4.2, Eq. dctdiag), computed on the host.
void dct2_matrix(int L, double* C);
void neumann_eigs(int L, double h, double* lam);

// Host-side DCT tables that depend on a grid's geometry alone: the DCT-II
// matrices along ax1 and ax2 (FP64 and FP32) and, when asked for, their
// arrangements for the per-axis tensor-core passes (tc) and the on-chip
// z-step (zs).  Computed once and kept for the last eight geometries of the
// process (rebuilding them, 65,536 cosines for a 256-face axis and then the
// arranged copies, took longer than many iterations of a solve).
struct HostTables {
    long long key[8];
    std::vector<double> C1, C2;
    std::vector<float> C1f, C2f;
    std::vector<float> tc[4], tn[4];   // per pass (empty where unused)
    std::vector<unsigned char> zs;
};
std::shared_ptr<const HostTables> host_tables(const int F[3], int ax1, int ax2, int pe, bool tc, bool zs);

// Device-side layout of a workspace for one volume.
struct Plan {
    Geometry G;
    int prec;                 // SAC_F64 / SAC_MIXED
    int W, K, RLf;            // line kernels: lines per CTA, faces per lane, smem row
    int seg_S, seg_G;          // b-step segment kernel: faces per segment (0: off), warps
    long long seg_tiles;       // its tiles of seg_lines() lines
    long long line_tiles, pass_tiles[4], elem_blocks;
    int use_tc;                // tensor-core z-step passes
    long long tc_tiles[4];
    long long admm_blocks;     // ADMM update blocks (tensor-core z-step)
    long long tc_floats[4];
    long long tn_floats[4];    // tensor-memory DCT operands (axes of at most 128 faces)
    TcCfg tc_cfg[4];           // ring / accumulator layout of each tensor-core pass
    TcCfg tc_cfg12;            // passes 1 and 2 in one launch (valid when fuse12)
    int fuse12;
    int use_zs;                // the z-step and dual update on the chip (zstep_slab.cu)
    long long zs_slabs, zs_bytes;
    ZsCfg zs_cfg;
    int rcap;
    int tables_up;            // the DCT tables of this plan are in ws (plan_upload)
    // device pointers inside ws
    Job* d_job;
    long long* d_pref_line;
    long long* d_pref_pass[4];
    long long* d_pref_elem;
    long long* d_pref_tc[4];
    long long* d_pref_admm;   // blocks of the ADMM update after the tensor-core passes
    long long* d_pref_seg;    // tiles of the b-step segment kernel
    long long* d_pref_zs;     // slabs of the on-chip z-step
    unsigned char* d_Czs;     // its split FP16 DCT operands
    float* d_Ctc[4];
    float* d_Ctn[4];
    void* d_tmaps;            // tensor maps of the tensor-core passes
    float* d_scale;
    int* d_status;
    int* d_rcount;
    unsigned long long* d_rlist;
    double* d_out;            // 64 doubles of reduction results
    double* d_part;
    long long n_part;
    double *d_C1, *d_C2, *d_lam1, *d_lam2;
    float *d_lam1f, *d_lam2f;   // FP32 copies (rebuilding the scale table after a change of rho)
    float *d_C1f, *d_C2f;
    double* arr[10];          // face-sized scratch arrays (8 bytes per face each)
    size_t bytes;             // total workspace bytes used
};

// plan layout; with ws == NULL only computes plan->bytes
int plan_layout(const sac_grid* g, const sac_params* p, void* ws, Plan* plan);
// upload the job descriptor, prefixes and (on the plan's first upload) the
// DCT tables (stream-ordered)
int plan_upload(Plan* plan, const sac_params* p, const void* I1, const void* I2, void* b, void* z, void* u,
                void* t1, void* t2, cudaStream_t st);
// line-launch description for this plan
LineLaunch plan_line_launch(const Plan* plan, int n_sqp, double near_bound, cudaStream_t st);

}  // namespace sac
