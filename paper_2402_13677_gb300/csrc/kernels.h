// Host launchers of the EBIT kernels (one translation unit per group).
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace ebit {

// interface.cu (FP64, no FMA contraction)
// validation of an uploaded interface; err (device, zeroed by the caller): bit 0 a colour other
// than 0/1, bit 1 a cut edge with a fraction outside [FMIN, 1 - FMIN]; uncut fractions set to 0
void launch_check_interface(const Grid& g, const uint8_t* vcol, double* hpos, double* vpos, int* err,
                            cudaStream_t st);
void launch_reconstruct(const Grid& g, const uint8_t* vcol, const double* hpos, const double* vpos, uint16_t* cseg,
                        uint8_t* flags, double* vf, cudaStream_t st);
void launch_band(const Grid& g, const uint16_t* cseg, const double* hpos, const double* vpos, uint8_t* flags,
                 double2* nb, cudaStream_t st);
// the same over the listed cells (reconstruction) and the listed cells with their neighbours (band)
void launch_reconstruct_list(const Grid& g, const int* list, const int* count, const uint8_t* vcol,
                             const double* hpos, const double* vpos, uint16_t* cseg, uint8_t* flags, double* vf,
                             cudaStream_t st);
void launch_band_list(const Grid& g, const int* list, const int* count, const uint16_t* cseg, const double* hpos,
                      const double* vpos, uint8_t* flags, double2* nb, cudaStream_t st);
void launch_sweep(const Grid& g, int axis, double dth, const int* list, const int* count, const uint8_t* vcol,
                  const double* hpos, const double* vpos, const uint16_t* cseg, const double2* uG, double* hdisp,
                  double* vdisp, uint8_t* vcol_n, double* hpos_n, double* vpos_n, int* status, cudaStream_t st);
// the cells within two of a cut cell (from the narrow-band list), their marks cleared after use
void launch_band_dilate(const Grid& g, const int* band, const int* nband, int* mark, int* list, int* count,
                        cudaStream_t st);
void launch_band_unmark(const Grid& g, const int* list, const int* count, int* mark, cudaStream_t st);
void launch_ug_list(const Grid& g, const Phys& p, const int* list, const int* count, const uint8_t* flags,
                    const double2* u_l, const double2* u_v, const double* mdot, const double2* nb, double2* uG,
                    cudaStream_t st);
void launch_energy_operator(const Grid& g, const Phys& p, const uint8_t* flags, const uint16_t* cseg,
                            const double* hpos, const double* vpos, const double* Ts_l, const double* Ts_v,
                            double* cd, double* dd, double* wl, double* wb, double* b, double* x0, cudaStream_t st);
void launch_curvature(const Grid& g, const uint8_t* flags, const uint16_t* cseg, const double* hpos,
                      const double* vpos, double* kap, cudaStream_t st);
void launch_mass_flux(const Grid& g, const Phys& p, const uint16_t* cseg, const double* hpos, const double* vpos,
                      const double* T_l, const double* T_v, double* mdot, cudaStream_t st);

// fields.cu
// f32w: WENO3 nonlinear weights in FP32 (mixed-precision mode)
void launch_advect_T(const Grid& g, const Phys& p, const uint8_t* flags, const double* T_l, const double* T_v,
                     const double2* u_l, const double2* u_v, double* Ts_l, double* Ts_v, cudaStream_t st);
void launch_compact(const Grid& g, const uint8_t* flags, int N, uint8_t mask, int* list, int* count, int* idxmap,
                    cudaStream_t st);
void launch_extend(const Grid& g, int mode, int iters, const int* list, const int* count, const uint8_t* flags,
                   const int* idxmap, const double2* nb, double* f, double* va, double* vb, cudaStream_t st);
// modes 0 and 1 (T_l into the vapour band, T_v into the liquid band) in one launch per sweep;
// ext[0..1] and ext[2..3] are the two ping-pong pairs
void launch_extend_T(const Grid& g, int iters, const int* list, const int* count, const uint8_t* flags,
                     const int* idxmap, const double2* nb, double* T_l, double* T_v, double* const ext[4],
                     cudaStream_t st);
void launch_split_T(const Grid& g, const uint8_t* flags, const double* x, const double* Ts_l, const double* Ts_v,
                    double* T_l, double* T_v, cudaStream_t st);
void launch_ghost_velocity(const Grid& g, const Phys& p, const int* band_list, const int* band_count,
                           const uint8_t* flags, const double* mdot, const double2* nb, const uint8_t* vcol,
                           const double* hpos, const double* vpos, double2* u_l, double2* u_v, double* ufx_l,
                           double* ufx_v, double* ufy_l, double* ufy_v, cudaStream_t st);
void launch_visc_operator(const Grid& g, const Phys& p, const double* vf, double* cd0, double* dd0, double* wl0,
                          double* wb0, double* cd1, double* dd1, double* wl1, double* wb1, cudaStream_t st);
void launch_mom_rhs(const Grid& g, const Phys& p, const double* vf, const double2* u_l, const double2* u_v,
                    const double2* gc, double2* bx, double2* by, double2* xx, double2* xy, cudaStream_t st);
void launch_ustar(const Grid& g, const Phys& p, const double2* sx, const double2* sy, const double2* gc,
                  const double* kap, const double* vf, double2* us_l, double2* us_v, double* fx_l, double* fx_v,
                  double* fy_l, double* fy_v, cudaStream_t st);
void launch_poisson_operator(const Grid& g, const Phys& p, const double* vf, const uint8_t* flags,
                             const uint16_t* cseg, const double* hpos, const double* vpos, const double* mdot,
                             const double* fx_l, const double* fx_v, const double* fy_l, const double* fy_v,
                             double* cd, double* dd, double* wl, double* wb, double* b, cudaStream_t st);
// ax/ay: face-acceleration scratch (x-faces ny*(nx+1), y-faces (ny+1)*nx); face velocities
// are updated when fx_l != null
// wl_p / wb_p: the Poisson operator's face weights dt / rho_f of the same volume fractions (they
// replace the per-face division), or null
void launch_project(const Grid& g, const Phys& p, const double* P, const double* vf, const double* kap,
                    const double* wl_p, const double* wb_p, double* ax, double* ay, double* fx_l, double* fx_v,
                    double* fy_l, double* fy_v, double2* gc, const double2* us_l, const double2* us_v, double2* u_l,
                    double2* u_v, cudaStream_t st);
int diag_blocks(const Grid& g);
void launch_diagnostics(const Grid& g, const Phys& p, const double* vf, const uint16_t* cseg, const double* hpos,
                        const double* vpos, const double* mdot, const uint8_t* flags, const double* fx_l,
                        const double* fx_v, const double* fy_l, const double* fy_v, const double* T_l,
                        const double* T_v, double* partial, unsigned* ticket, double* clock, double* out,
                        cudaStream_t st);

}  // namespace ebit
