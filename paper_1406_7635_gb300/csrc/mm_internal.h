// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda.h>   // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace mm {

constexpr int kRegions = 256;
// cell code: the region index of a cell that carries a magnetisation (mask
// set, Msat > 0), kVacuum otherwise; the exchange table has a zero column at
// kVacuum, so a vacuum neighbour contributes nothing without a branch
constexpr int kVacuum = kRegions;
constexpr int kXStride = kRegions + 1;   // row length of the exchange table
constexpr int kHistCap = 1 << 20;   // accepted-step sizes kept for replay

#ifdef __CUDACC__
// Waits until the preceding kernel of the stream has completed and its writes
// are visible (no-op for a kernel launched without the attribute), then lets
// the next kernel's blocks be scheduled once every block of this one has
// passed this point.
__device__ __forceinline__ void grid_dependency_wait() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}
#endif

// Per-region parameters, float32, derived on the host from mm_material
// (Sec. II.A: 256-entry look-up tables indexed by the region byte).
struct RegionLUT {
  float msat[kRegions];
  float alpha[kRegions];
  float gfac[kRegions];   // -gamma / (1 + alpha^2)   (Eq. eqLLG, damping sign)
  float k1[kRegions];     // 2 Ku1 / Msat            (uniaxial field, Ku1 part)
  float k2[kRegions];     // 4 Ku2 / Msat            (uniaxial field, Ku2 part)
  float u[3][kRegions];   // anisotropy axis
  float b0[3][kRegions];  // B_ext = b0 + b1 sin(2 pi f t + phase)
  float b1[3][kRegions];
  float dmi[kRegions];    // 2 D / Msat                (interfacial DMI field)
  float dbc[kRegions];    // D / (2 Aex)              (boundary derivative; 0 if Aex = 0)
};

// Per-region spin-transfer-torque parameters (Sec. III, Zhang-Li and
// Slonczewski torques), float32, derived on the host from mm_material.
struct SttLUT {
  float zlu[3][kRegions]; // Zhang-Li velocity mu_B j / (2 e Msat (1 + xi^2)) (m/s)
  float zla[kRegions];    // (1 + xi alpha) / (1 + alpha^2)
  float zlb[kRegions];    // (xi - alpha) / (1 + alpha^2)
  float slg[kRegions];    // gamma beta / (1 + alpha^2), beta = j_z hbar / (Msat e d)
  float slp[kRegions];    // P Lambda^2
  float sl1[kRegions];    // Lambda^2 + 1
  float sl2[kRegions];    // Lambda^2 - 1
  float sle[kRegions];    // eps'
  float mp[3][kRegions];  // fixed-layer direction
  float alpha[kRegions];  // damping (the Slonczewski field-like mixing)
};

// Spin-transfer torques of a context: which are on, their table, and the
// central-difference factors 1 / (2 Delta) of the Zhang-Li gradient.
struct Stt {
  int zl, sl;
  const SttLUT* lut;
  float hx, hy, hz;
};

// Grid and padded-FFT geometry.
struct Geom {
  int nx, ny, nz;
  long long n;            // nx * ny * nz
  float idx2, idy2, idz2; // 1 / d^2 per axis
  int px, py, pz;         // padded sizes (power of two >= 2n - 1; 1 if n == 1)
  int lx;                 // complex length of the x transform (px / 2, or 1)
  int hx;                 // spectrum columns kept along x: lx + 1 (or 1)
  int hxs;                // row stride of the spectrum buffer (complex)
  int srows;              // rows per plane in the spectrum buffer (py if pz > 1 else ny)
  long long sc;           // complex elements per component of the spectrum buffer
  int hkx, hky, hkz;      // octant sizes of the kernel spectrum
  // fused path (fft_fused.cu): spectrum laid out [3][hx][nz][ny], one
  // cluster of cly*clz blocks per kx plane, each transforming ly x lz points
  int fused, cly, clz, ly, lz;
  int xrows;              // x-row kernels: rows per block (0 = default rule)
  float cdx, cdy;         // cell sizes along x and y (DMI ghost values)
  int pbcx, pbcy, pbcz;   // periodic images on each side (0 = open axis)
};

// Programmatic dependent launch of the RK stage kernels: a kernel launched
// with it may start on free SMs while its predecessor drains, and waits for
// the predecessor's results with grid_dependency_wait() before reading them.
// With the cluster (y, z) kernel, per geometry, from same-GPU measurements
// (ms per step, none / row / y-z / both): 128 x 128 x 32 (z-split y/z kernel,
// 1.7 waves of large blocks) 0.549 / 0.535 / 0.549 / 0.550; 256 x 256 x 1 film
// (one wave) 0.165 / 0.197 / 0.161 / 0.203.  The register-resident (y, z)
// kernels of fft_yz3.cu are always dependents; behind the one-kernel 2-D path
// the context also makes the row kernel one (launch_rowstage's `dep`).
inline bool pdl_row(const Geom& g) { return g.fused && g.clz == 2; }
inline bool pdl_yz(const Geom& g) { return !pdl_row(g); }

// Integrator state on the device (one per context).  Every kernel of a step
// reads it, so a captured graph of one attempt can be replayed unchanged.
struct DevState {
  double t, dt, h;          // time, proposed step, step of the current attempt
  double t_end;             // run() target
  double max_err, headroom, dt_min, dt_max;
  double last_err;
  double stage_t[7];        // t + c_s h
  long long accepted, rejected, evals;
  long long target;         // steps(): stop at this accepted count
  int mode;                 // 0 steps(n), 1 run(t_end), 2 replay
  int parity;               // which m / k1 buffers are current (FSAL swap)
  int done;                 // 1: no more attempts in this call
  int status;               // MM_OK or an error code
  int fixed_idx, fixed_n;   // replay cursor
  int hist_n;
  unsigned int err_bits;    // max step error of this attempt (float bits)
  unsigned int ticket;      // last-block election in the error kernel
  int call_attempts;         // attempts since the last begin
  int precession;
  int method;               // 0 Dormand-Prince RK45, 1 Bogacki-Shampine RK23
  long long wait_cycles;    // limit of a kernel's wait on its tensor copies (SM clock cycles)
};

// default wait limit: 2^30 cycles, about half a second at the maximum SM clock
constexpr long long kWaitCycles = 1LL << 30;

struct Buffers {
  float* m[2];        // current / candidate m (parity)
  float* k[7];        // RK stages; k[0] and k[6] swap roles with parity
  float* ms;          // stage input m_s (even stages of the row-stage path)
  float* ms2;         // odd-stage inputs of the row-stage path
  float* bd;          // demag field
  float2* spec;       // spectrum work buffer
  float* kt;          // kernel spectrum octant [6][hkz][hky][hkx]
  float* ktf;         // fused path: the same octant as [hkx][6][hkz][hky]
  float2* tw;         // twiddles W[k] = exp(-2 pi i k / 2048)
  uint8_t* mask;
  uint8_t* region;
  RegionLUT* lut;
  float* xlut;        // [256][257]: 2 S H(Aex/Msat) exchange couplings, column 256 = 0
  int* code;          // per cell: region, or kVacuum
  DevState* st;
  double* hist;       // accepted step sizes
  double* fixed;      // replay sequence
  double* acc;        // energy accumulators
  float* out;         // field/torque output for getters
  float* part;        // row-stage path: the earlier-stage sums of a row kernel (k_rs_partial)
};

// enabled field terms; dmi is set by the library when a region has D != 0
struct Terms { int demag, exch, anis, zeeman, dmi; };

// pbc (may be null): periodic images per axis; a periodic axis is not padded
Geom make_geom(int nx, int ny, int nz, double dx, double dy, double dz, const int* pbc = nullptr);

// Instance dimension of the fused convolution kernels: `count` instances of
// one grid laid out back to back; optional per-instance Msat (every cell
// magnetic) and a per-instance done flag read at done[i * done_stride].
struct BatchArgs {
  int count;
  const float* msat;
  const int* done;
  int done_stride;
};

// sets the message mm_last_error() returns on this thread
void set_last_error(const std::string& msg);
// grid and padded-FFT geometry (fused fields left zero; see fused_plan)
struct Geom;


// ---- launch wrappers (stream-ordered) ----
// demag convolution of M = Msat m (m = `m`), result in b.bd
void launch_demag(const Geom& g, const Buffers& b, const float* m, cudaStream_t s);
// fused three-kernel convolution; fused_plan() decides whether g supports it
bool fused_plan(Geom& g);
// tile choices of the fused convolution for g (an autotuner times them):
// residue splits (cly, clz) that satisfy the plan's limits, and rows per
// block of the x-row kernels; return the number written (at most max)
int fused_splits(const Geom& g, int (*out)[2], int max);
int fused_xrows(const Geom& g, int* out, int max);
// applies a split chosen from fused_splits
void fused_set_split(Geom& g, int cly, int clz);
void launch_demag_fused(const Geom& g, const Buffers& b, const float* m, cudaStream_t s);
void launch_demag_fused_batch(const Geom& g, const Buffers& b, const float* m, cudaStream_t s, const BatchArgs& ba);
void launch_kt_transpose(const Geom& g, const float* kt, float* ktf, cudaStream_t s);
// only the (y, z) part of the fused convolution (k_yz), spectrum in place
void launch_demag_yz(const Geom& g, const Buffers& b, cudaStream_t s);
// The three-kernel (y, z) part (fft_yz3.cu): y forward into T (yz3_bytes(g)
// bytes, [kx][c][z][ky]), the column kernel (z, kernel product, z inverse)
// in place in T, y inverse back into the spectrum; yz3_plan(g) tells whether
// the grid supports it.  launch_demag_fused3: the whole convolution with it.
bool yz3_plan(const Geom& g);
// 2-D grids: y forward, kernel product and y inverse of a kx plane in one
// block (fft_yz3.cu), in place in the spectrum; y2d_plan(g) tells whether
// the grid supports it.  launch_demag_fused2d: the whole convolution with it.
bool y2d_plan(const Geom& g);
void launch_demag_y2d(const Geom& g, const Buffers& b, cudaStream_t s);
void launch_demag_fused2d(const Geom& g, const Buffers& b, const float* m, cudaStream_t s);
size_t yz3_bytes(const Geom& g);
void launch_demag_yz3(const Geom& g, const Buffers& b, float2* T, cudaStream_t s);
void launch_demag_fused3(const Geom& g, const Buffers& b, const float* m, float2* T, cudaStream_t s);
// one of the three kernels of launch_demag_yz3 (0 y forward, 1 column
// kernel, 2 y inverse), for per-kernel timing
void launch_yz3_part(const Geom& g, const Buffers& b, float2* T, int part, cudaStream_t s);
// Tensor maps of the row-stage kernels' TMA path (rowstage.cu): the spectrum
// [3][hx][nz][ny] (8-byte elements) with box (ROWS, 1, L + 1, 3), the stage
// inputs [3][nz][ny][nx] with boxes (L, ROWS + 2, 1, 1) (own plane and the
// two halo rows) and (L, ROWS, 1, 1) (neighbour planes), and the cell codes
// [nz][ny][nx] with the same two boxes.  ok_spec / ok_sten = 0: the spectrum
// / stencil rows take the cp.async path.
struct RsMaps {
  CUtensorMap spec;
  CUtensorMap ms_own, ms_pl, ms2_own, ms2_pl;
  CUtensorMap code_own, code_pl;
  int ok_spec, ok_sten;
};
// fills *m for this grid and its buffers (a flag stays 0 when its copies do
// not apply or the driver's encoder is unavailable)
void rowstage_maps(const Geom& g, const Buffers& b, RsMaps* m);

// fused RK45 stage kernels (rowstage.cu): kind 0 = stage-input prep of stage
// s, kind 1 = row kernel of stage s (mode 0 first stage only, 1 next stage,
// 2 last stage with error and controller); maps from rowstage_maps.  With
// b.part set, the row kernels of modes 1 and 2 read their earlier-stage sums
// from it: launch_rs_partial for the same (s, mode) must complete first.
void launch_rowstage(const Geom& g, const Buffers& b, const Terms& T, const RsMaps& maps, int kind, int s, int mode,
                     double freq, double phase, cudaStream_t st, bool dep = false);
// the earlier-stage sums of the row kernel of stage s into b.part: mode 1
// m + sum_{j<s} a_{s+1,j} k_j, mode 2 sum_{j<6} e_j k_j (needs k_0 .. k_{s-1})
void launch_rs_partial(const Geom& g, const Buffers& b, int s, int mode, cudaStream_t st);
// kernel spectrum octant: fills b.kt (float64 work inside); returns cudaError
cudaError_t build_kernel_spectrum(const Geom& g, double dx, double dy, double dz, float* kt,
                                  cudaStream_t s);
// kernel precompute on caller-provided work space (no allocation, no host
// round trips); sizes of the work areas in doubles
size_t kernel_work_doubles(const Geom& g);
size_t kernel_table_doubles(const Geom& g);
cudaError_t build_kernel_spectrum_ws(const Geom& g, double dx, double dy, double dz, float* kt, double* w0,
                                     double* w1, double* tab, cudaStream_t s);
cudaError_t demag_tensor_offsets(int n, const int32_t* d_off, double dx, double dy, double dz,
                                 double* d_out, cudaStream_t s);

// RK45 pieces (llg.cu).  DevState is followed in the same allocation by the
// per-attempt stage coefficients; devstate_bytes() is the allocation size.
size_t devstate_bytes();
// mode 0: steps(nsteps); 1: run(t_end); 2: replay of the fixed sequence
void launch_begin_mode(const Buffers& b, int mode, long long nsteps, double t_end, cudaStream_t s);
void launch_stage_input(const Geom& g, const Buffers& b, int stage, cudaStream_t s);
// torque of stage `stage` (0..6) at m_s (stage 0: the current m), into the
// k buffer holding that stage's role
// (plus the spin-transfer torques S where switched on)
void launch_torque_t(const Geom& g, const Buffers& b, const Terms& T, const Stt& S, int stage, double freq,
                     double phase, cudaStream_t s);
void launch_error_control(const Geom& g, const Buffers& b, cudaStream_t s);
void launch_copy_mcur(const Geom& g, const Buffers& b, float* dst, cudaStream_t s);
// getters at m, time st->t: mode 0 B_eff -> b.out, 1 torque -> b.out,
// 2 energy sums -> b.acc, 4 max |torque| -> b.acc[0] (torques with S)
void launch_field_out_t(const Geom& g, const Buffers& b, const Terms& T, const Stt& S, const float* m, int mode,
                        double freq, double phase, cudaStream_t s);
void launch_normalize(const Geom& g, const Buffers& b, float* m, cudaStream_t s);
// *flag = 1 if the 3 n floats of a and b differ in any bit (caller zeroes it)
void launch_m_differs(const Geom& g, const float* a, const float* b, int* flag, cudaStream_t s);
// cell codes from mask, region and the Msat table
void launch_codes(const Geom& g, const Buffers& b, cudaStream_t s);
// sets the launch attributes (dynamic shared memory) of the row-stage
// kernels this grid uses; call outside stream capture
cudaError_t prepare_rowstage(const Geom& g);

// FNO surrogate (fno.cu)
}  // namespace mm
struct mm_fno;
namespace mm {
void launch_fno_demag(mm_fno* f, const Geom& g, const Buffers& b, const float* m, float inv_ref, float mu0_ref,
                      float* bd, cudaStream_t s);
void launch_rel_err(long long n, const float* a, const float* b, double* acc, cudaStream_t s);
bool fno_matches(mm_fno* f, const Geom& g);
void launch_to_u(const Geom& g, const Buffers& b, const float* m, float inv_ref, float* u, cudaStream_t s);
void launch_scale(long long n, const float* x, float a, float* y, cudaStream_t s);
}  // namespace mm
