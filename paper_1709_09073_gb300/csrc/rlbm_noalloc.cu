// rlbm_step_noalloc: the FP64 fused stream-collide step for one small domain,
// with every byte of working memory in one fixed file-scope device array.
//
// Some callers cannot call cudaMalloc: a host application whose own allocator
// has already reserved the device memory and hands out nothing else, or code on
// a latency-critical path where cudaMalloc/cudaFree are banned because they can
// synchronise the whole device. They still own their inputs and outputs (a
// population checkpoint in, one out); this entry point keeps its halo-padded
// ping-pong copies, domain descriptor, tile list and status word in g_scratch
// below, so the call itself allocates nothing.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the status word is cleared at the start of each call, everything
// else is overwritten before it is read. Calls whose work overlaps on the GPU
// race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "rlbm.h"
#include "rlbm_common.h"
#include "rlbm_launch.h"

using namespace rlbm;

namespace {

constexpr size_t kScratchBytes = RLBM_NOALLOC_SCRATCH_BYTES;
constexpr size_t kAlignB = 256;
constexpr int kMaxDevices = 64;

// The scratch array. The CUDA runtime reserves it on a device when this
// module is loaded there and holds it until the process exits. In host code
// `g_scratch` is only a host-side stand-in for the symbol, never a device
// address: the address is looked up with cudaGetSymbolAddress per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch, per device ordinal

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool bc_ok(int b) {
  return b == RLBM_PERIODIC || b == RLBM_ZERO_GRADIENT || b == RLBM_FIXED_T_WALL || b == RLBM_VELOCITY_WALL;
}

// Offsets (bytes) of the pieces inside g_scratch for one domain.
struct ScratchPlan {
  DomDev D;
  int ntiles, tiles_x;
  size_t dom_off, tiles_off, pop_off[2], total;
};

int check_domain(const rlbm_domain* d, int edf) {
  if (!d || edf < RLBM_MJ || edf > RLBM_BE) return RLBM_E_ARG;
  if (d->nx < 1 || d->ny < 1 || !(d->tau > 0.0)) return RLBM_E_ARG;
  if (!bc_ok(d->bc_xlo) || !bc_ok(d->bc_xhi) || !bc_ok(d->bc_ylo) || !bc_ok(d->bc_yhi)) return RLBM_E_ARG;
  if ((d->bc_xlo == RLBM_PERIODIC) != (d->bc_xhi == RLBM_PERIODIC)) return RLBM_E_ARG;
  if ((d->bc_ylo == RLBM_PERIODIC) != (d->bc_yhi == RLBM_PERIODIC)) return RLBM_E_ARG;
  const int bc[4] = {d->bc_xlo, d->bc_xhi, d->bc_ylo, d->bc_yhi};
  const double tw[4] = {d->t_wall_xlo, d->t_wall_xhi, d->t_wall_ylo, d->t_wall_yhi};
  bool vw = false;
  double tvw = 0.0;
  for (int k = 0; k < 4; ++k) {
    if ((bc[k] == RLBM_FIXED_T_WALL || bc[k] == RLBM_VELOCITY_WALL) && !(tw[k] > 0.0)) return RLBM_E_ARG;
    if (bc[k] == RLBM_VELOCITY_WALL) {
      if (vw && tw[k] != tvw) return RLBM_E_ARG;
      vw = true;
      tvw = tw[k];
    }
  }
  if (vw && !(d->n_wall > 0.0)) return RLBM_E_ARG;
  if (!(d->accel_x > -1.0 && d->accel_x < 1.0 && d->accel_y > -1.0 && d->accel_y < 1.0)) return RLBM_E_ARG;
  if (!(d->eta_s >= 0.0) || !(d->eta_s < 1e300)) return RLBM_E_ARG;  // as rlbm_create checks it
  return RLBM_OK;
}

// Lay one FP64 domain out inside the scratch array: status word, descriptor,
// tile list, two population copies (blocks of 32 cells, halo ring included,
// the library's layout). Returns RLBM_E_SCRATCH if it does not fit.
int plan_scratch(const rlbm_domain* d, ScratchPlan& P) {
  // any side beyond 2^20 cells is far past the limit; this also bounds the arithmetic below
  if (d->nx > (1 << 20) || d->ny > (1 << 20)) return RLBM_E_SCRATCH;
  DomDev& D = P.D;
  D = DomDev{};
  D.nx = d->nx;
  D.ny = d->ny;
  D.nblk = blocks_per_row(d->nx);
  D.pitch = (long long)D.nblk * kBlk;
  D.off = 0;
  D.bc[0] = d->bc_xlo; D.bc[1] = d->bc_xhi; D.bc[2] = d->bc_ylo; D.bc[3] = d->bc_yhi;
  D.inv_tau = 1.0 / d->tau;
  D.t_wall[0] = d->t_wall_xlo; D.t_wall[1] = d->t_wall_xhi;
  D.t_wall[2] = d->t_wall_ylo; D.t_wall[3] = d->t_wall_yhi;
  D.ref_n = D.ref_theta = D.scale = 1.0;  // used by the mixed storages only
  D.order = 5;
  D.eta_s = d->eta_s > 0.0 ? d->eta_s : 0.0;
  D.tau = d->tau;
  D.accel_x = d->accel_x;
  D.accel_y = d->accel_y;
  D.n_wall = d->n_wall;
  P.tiles_x = (d->nx + kTileW - 1) / kTileW;
  P.ntiles = P.tiles_x * ((d->ny + kTileH - 1) / kTileH);
  size_t b = kAlignB;  // [0, 256): status word
  P.dom_off = b;
  b = round_up(b + sizeof(DomDev), kAlignB);
  P.tiles_off = b;
  b = round_up(b + sizeof(Tile) * (size_t)P.ntiles, kAlignB);
  const size_t pop_bytes = round_up((size_t)(d->ny + 2) * (size_t)D.pitch * sizeof(double), kAlignB);
  P.pop_off[0] = b;
  P.pop_off[1] = b + pop_bytes;
  P.total = b + 2 * pop_bytes;
  return P.total <= kScratchBytes ? RLBM_OK : RLBM_E_SCRATCH;
}

// Device address of g_scratch on the current device. The first call on a
// device looks it up and opts the FP64 kernels into their shared memory.
int scratch_address(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RLBM_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return RLBM_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return RLBM_E_CUDA;
    if (prepare_f64() != cudaSuccess) return RLBM_E_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<char*>(g_scratch_addr[dev]);
  return RLBM_OK;
}

// Write the descriptor and the tile list into the scratch array and clear the
// status word (it keeps the previous call's bits otherwise).
__global__ void k_noalloc_setup(DomDev D, DomDev* d_dom, Tile* tiles, int ntiles, int tiles_x,
                                unsigned* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    *d_dom = D;
    *status = 0u;
  }
  if (t < ntiles) tiles[t] = Tile{0, (t % tiles_x) * kTileW, (t / tiles_x) * kTileH, 0};
}

}  // namespace

extern "C" int rlbm_step_noalloc(const rlbm_domain* domain, int edf, int nsteps, const double* f_in,
                                 double* f_out, void* cuda_stream, unsigned* warnings) {
  int r = check_domain(domain, edf);
  if (r) return r;
  if (nsteps < 0 || !f_in || !f_out) return RLBM_E_ARG;
  ScratchPlan P;
  if ((r = plan_scratch(domain, P))) return r;
  char* base = nullptr;
  if ((r = scratch_address(&base))) return r;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned* d_status = reinterpret_cast<unsigned*>(base);
  DomDev* d_dom = reinterpret_cast<DomDev*>(base + P.dom_off);
  Tile* d_tiles = reinterpret_cast<Tile*>(base + P.tiles_off);
  void* pop[2] = {base + P.pop_off[0], base + P.pop_off[1]};

  k_noalloc_setup<<<(P.ntiles + 255) / 256, 256, 0, s>>>(P.D, d_dom, d_tiles, P.ntiles, P.tiles_x, d_status);
  cudaError_t e = cudaGetLastError();
  CopyArgs ca;
  ca.doms = d_dom;
  ca.dom = 0;
  ca.q0 = 0;
  ca.nq = 72;
  if (e == cudaSuccess) {  // checkpoint layout -> halo-padded copy 0
    ca.to_dense = 0;
    ca.pop = pop[0];
    ca.dense = const_cast<double*>(f_in);
    e = launch_copy_f64(ca, s);
  }
  int cur = 0;
  for (int i = 0; i < nsteps && e == cudaSuccess; ++i) {
    StepArgs a;
    a.doms = d_dom;
    a.tiles = d_tiles;
    a.ntiles = P.ntiles;
    a.fin = pop[cur];
    a.fout = pop[1 - cur];
    a.status = d_status;
    a.tmaps = nullptr;
    a.variant = 0;
    a.wait_ns = 0;
    a.halo = 2;
    e = launch_step_f64(edf, a, P.ntiles, s);
    cur = 1 - cur;
  }
  if (e == cudaSuccess) {  // halo-padded copy -> checkpoint layout
    ca.to_dense = 1;
    ca.pop = pop[cur];
    ca.dense = f_out;
    e = launch_copy_f64(ca, s);
  }
  if (e == cudaSuccess && warnings) {
    e = cudaMemcpyAsync(warnings, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  return e == cudaSuccess ? RLBM_OK : RLBM_E_CUDA;
}
