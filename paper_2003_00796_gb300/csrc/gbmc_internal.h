// gbmc_internal.h -- host-side structures of the library (tables, context) and
// the launch wrappers of the kernels.
#pragma once

#include <string>
#include <vector>

#include "gbmc_common.cuh"

namespace gb {

// FP32 tables and their grids, built on the host in FP64.
struct Tables {
  int n_mat = 0, nE = 0, nR = 0, nA = 0;
  double emin = 0.0, emax = 0.0;
  float lg0 = 0.f, inv_d = 0.f;
  float lr0[GBMC_MAX_MAT][2] = {}, inv_dr[GBMC_MAX_MAT][2] = {};
  float la0 = 0.f, inv_da = 0.f;
  int off_major = 0, off_soft = 0;   // offsets in data
  std::vector<float> data;         // photon region (tab_off of Q_MU_*, majorant),
                                   // charged region (other quantities, soft A',
                                   // element CDFs): see tab_off_e
  int n_staged = 0;                // floats of data before the element CDF rows
  int off_el[GBMC_MAX_MAT] = {};   // element CDF rows of material m in data (-1: one element)
  int off_mpar = 0;                // per-material parameter block (MatPar) in data
  std::vector<double> mu_tot;      // FP64 total attenuation per material and node
  DevMat dmat[GBMC_MAX_MAT];
};

bool build_tables(Tables& T, const gbmc_material* mats, int n_mat, const gbmc_transport& tp,
                  double emax, int nE, int nA);
void build_majorant(Tables& T, const double* rho_max);
void majorant_table(const Tables& T, const double* rho_max, float* out);   // T.nE floats

namespace host {
double electron_density(const gbmc_material& m);
double sigma_kn(double k);
double rayleigh_int(double b);
void photon_xs(const gbmc_material& m, double E, double* co, double* pe, double* ray, double* pair);
double s_col(const gbmc_material& m, bool pos, double T);
double s_restricted(const gbmc_material& m, bool pos, double T, double wcc, double wcr);
double soft_aprime(double mbar);
}  // namespace host

// ---- kernel launch wrappers (defined in the .cu files) --------------------
size_t plain_smem_bytes(const DevProblem& P);
cudaError_t launch_adjoint(const DevProblem& P, const float* wv, int grid, int block, cudaStream_t s);
cudaError_t launch_adjoint_weights(const double* g, const float* rho, int64_t nvox, double vol,
                                   float* wv, cudaStream_t s);
cudaError_t launch_plain(const DevProblem& P, int grid, int block, cudaStream_t s, bool check = false);
cudaError_t launch_wavefront_pass(const DevProblem& P, bool photon, const WfRing& R,
                                  const PassState* ps, int grid, int block, int min_blocks,
                                  const float* wv, cudaStream_t s);
cudaError_t launch_knock_pass(const DevProblem& P, const WfRing& R, const PassState* ps, int grid,
                              int block, const float* wv, cudaStream_t s);
size_t drain_smem_bytes(const DevProblem& P);
cudaError_t launch_drain_pass(const DevProblem& P, const WfRing& R, const PassState* ps, int grid,
                              const float* wv, cudaStream_t s);
// in_graph = 1 only inside the body of the while loop whose condition handle is h
cudaError_t launch_pass_ctl(const PassCtl& c, PassState* ps, unsigned int* cnt, unsigned int* err,
                            int first, unsigned long long* loop, cudaStream_t s,
                            cudaGraphConditionalHandle h = 0, int in_graph = 0);
cudaError_t launch_flush_tiles(float* tiles, int64_t stride, int K, const double* inv_n,
                               double* s1, double* s2, double* dep, int sms, cudaStream_t s);
cudaError_t launch_first_interactions(const DevProblem& P, uint32_t hist0, int n, float* xyz,
                                      int* type, cudaStream_t s);
cudaError_t launch_finalize(const double* s1, const double* s2, const float* rho, int64_t nvox,
                            double n_hist, double k_batches, double voxel_volume, int dose,
                            double* mean, double* var, cudaStream_t s);
cudaError_t launch_flush_tiles_scalar(float* tiles, int64_t stride, int64_t nvox, int K,
                                      const double* inv_n, double* s1, double* s2, double* dep,
                                      int sms, cudaStream_t s);
cudaError_t launch_add_moments(double* s1, double* s2, const double* x1, const double* x2,
                               int64_t nvox, cudaStream_t s);
cudaError_t launch_batch_weights(double* inv_n, uint64_t n_hist, int K, cudaStream_t s);
cudaError_t launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                               uint32_t k1, uint32_t* out, int n, cudaStream_t s);
cudaError_t launch_validate_phantom(const uint8_t* mat, const float* rho, int64_t nvox, int n_mat,
                                    unsigned int* bad, float* rho_max, cudaStream_t s);

}  // namespace gb
