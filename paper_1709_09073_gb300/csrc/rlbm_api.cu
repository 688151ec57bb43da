// Host side of the C ABI declared in include/rlbm.h: workspace layout, handle,
// CUDA-graph replay of the step, host/device transfers and status handling.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "rlbm.h"
#include "rlbm_common.h"
#include "rlbm_launch.h"

using namespace rlbm;

namespace {

constexpr size_t kAlign = 256;
constexpr int kChunkPairs = 16;  // a chunk graph holds 2 * kChunkPairs steps

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t elem_size(int storage) {
  switch (storage) {
    case RLBM_F64: return 8;
    case RLBM_F32:
    case RLBM_F32DEV: return 4;
    case RLBM_BF16DEV:
    case RLBM_F16DEV: return 2;
    default: return 0;
  }
}

struct Layout {
  size_t esize = 0;
  size_t status_off = 0, doms_off = 0, tiles_off = 0, ptiles_off = 0, tmaps_off = 0, pop_off[2] = {0, 0};
  size_t pop_elems = 0, pop_bytes = 0, total = 0;
  std::vector<DomDev> dd;
  std::vector<Tile> tiles;   // kTileW x kTileH tiles: every kernel but the mixed L1 step
  std::vector<Tile> ptiles;  // the same with each domain's ragged last x block packed (Tile::w)
};

bool valid_bc(int b) {
  return b == RLBM_PERIODIC || b == RLBM_ZERO_GRADIENT || b == RLBM_FIXED_T_WALL || b == RLBM_VELOCITY_WALL ||
         b == RLBM_EXCHANGED;
}

int validate(const rlbm_config* c) {
  if (!c || c->ndomains < 1 || !c->domains) return RLBM_E_ARG;
  if (c->edf < RLBM_MJ || c->edf > RLBM_BE) return RLBM_E_ARG;
  if (!elem_size(c->storage)) return RLBM_E_ARG;
  if (c->order < 2 || c->order > 5 || (c->storage != RLBM_F64 && c->order != 5)) return RLBM_E_UNSUPPORTED;
  for (int i = 0; i < c->ndomains; ++i) {
    const rlbm_domain& d = c->domains[i];
    if (d.nx < 1 || d.ny < 1 || !(d.tau > 0.0)) return RLBM_E_ARG;
    if (!(d.eta_s >= 0.0) || !(d.eta_s < 1e300)) return RLBM_E_ARG;
    if (!valid_bc(d.bc_xlo) || !valid_bc(d.bc_xhi) || !valid_bc(d.bc_ylo) || !valid_bc(d.bc_yhi))
      return RLBM_E_ARG;
    // faces are exchanged along y only (rlbm_pack_edge_rows / rlbm_unpack_ghost_rows)
    if (d.bc_xlo == RLBM_EXCHANGED || d.bc_xhi == RLBM_EXCHANGED) return RLBM_E_ARG;
    if ((d.bc_xlo == RLBM_PERIODIC) != (d.bc_xhi == RLBM_PERIODIC)) return RLBM_E_ARG;
    if ((d.bc_ylo == RLBM_PERIODIC) != (d.bc_yhi == RLBM_PERIODIC)) return RLBM_E_ARG;
    const double tw[4] = {d.t_wall_xlo, d.t_wall_xhi, d.t_wall_ylo, d.t_wall_yhi};
    const int bc[4] = {d.bc_xlo, d.bc_xhi, d.bc_ylo, d.bc_yhi};
    double tvw = 0.0;
    bool vw = false;
    for (int k = 0; k < 4; ++k) {
      if ((bc[k] == RLBM_FIXED_T_WALL || bc[k] == RLBM_VELOCITY_WALL) && !(tw[k] > 0.0)) return RLBM_E_ARG;
      if (bc[k] == RLBM_VELOCITY_WALL) {
        if (vw && tw[k] != tvw) return RLBM_E_ARG;  // one theta_wall for all velocity walls
        vw = true;
        tvw = tw[k];
      }
    }
    if (vw && !(d.n_wall > 0.0)) return RLBM_E_ARG;
    if (!(d.accel_x > -1.0 && d.accel_x < 1.0 && d.accel_y > -1.0 && d.accel_y < 1.0)) return RLBM_E_ARG;
    if ((vw || d.accel_x != 0.0 || d.accel_y != 0.0) && c->storage != RLBM_F64) return RLBM_E_UNSUPPORTED;
    if (c->storage != RLBM_F64 && (!(d.scale > 0.0) || !(d.ref_n > 0.0) || !(d.ref_theta > 0.0)))
      return RLBM_E_ARG;
    if ((long long)d.nx * d.ny > (1LL << 31)) return RLBM_E_ARG;
  }
  return 0;
}

void make_layout(const rlbm_config* c, Layout& L) {
  L.esize = elem_size(c->storage);
  const size_t es = L.esize;
  size_t off = 0;  // elements
  long long foff = 0;  // cells before the domain in packed field arrays
  L.dd.resize(c->ndomains);
  L.tiles.clear();
  L.ptiles.clear();
  for (int i = 0; i < c->ndomains; ++i) {
    const rlbm_domain& d = c->domains[i];
    DomDev& D = L.dd[i];
    std::memset(&D, 0, sizeof(D));
    D.nx = d.nx;
    D.ny = d.ny;
    D.nblk = blocks_per_row(d.nx);
    D.pitch = (long long)D.nblk * kBlk;
    D.off = (long long)off;
    D.foff = foff;
    foff += (long long)d.nx * d.ny;
    D.bc[0] = d.bc_xlo; D.bc[1] = d.bc_xhi; D.bc[2] = d.bc_ylo; D.bc[3] = d.bc_yhi;
    D.inv_tau = 1.0 / d.tau;
    D.t_wall[0] = d.t_wall_xlo; D.t_wall[1] = d.t_wall_xhi;
    D.t_wall[2] = d.t_wall_ylo; D.t_wall[3] = d.t_wall_yhi;
    D.ref_n = d.ref_n > 0.0 ? d.ref_n : 1.0;
    D.ref_theta = d.ref_theta > 0.0 ? d.ref_theta : 1.0;
    D.scale = d.scale > 0.0 ? d.scale : 1.0;
    D.order = c->order;
    D.eta_s = d.eta_s;
    D.tau = d.tau;
    D.accel_x = d.accel_x;
    D.accel_y = d.accel_y;
    D.n_wall = d.n_wall;
    D.inv_tau_f = (float)D.inv_tau;
    D.eta_s_f = (float)D.eta_s;
    for (int k = 0; k < 4; ++k) D.t_wall_f[k] = (float)D.t_wall[k];
    off = align_up(off + (size_t)(d.ny + 2) * (size_t)D.pitch, kAlign / es);
    // row bands of tiles, in the same order in both lists; in the packed list a
    // ragged last block of w <= kPackMaxW cells becomes one tile per
    // kTileH * (32 / w) rows, placed after the first band it covers
    const int xl = (d.nx - 1) / kTileW * kTileW, wl = d.nx - xl;
    const int pw = wl <= kPackMaxW ? wl : 0;
    const int prow = kTileH * packed_rows_per_warp(pw);
    for (int y0 = 0; y0 < d.ny; y0 += kTileH) {
      for (int x0 = 0; x0 < d.nx; x0 += kTileW) {
        L.tiles.push_back(Tile{i, x0, y0, 0});
        if (x0 < xl || !pw) L.ptiles.push_back(Tile{i, x0, y0, 0});
        else if (y0 % prow == 0) L.ptiles.push_back(Tile{i, x0, y0, pw});
      }
    }
  }
  L.pop_elems = off;
  L.pop_bytes = align_up(off * es, kAlign);
  size_t b = 0;
  L.status_off = b;
  b += kAlign;
  L.doms_off = b;
  b = align_up(b + sizeof(DomDev) * L.dd.size(), kAlign);
  L.tiles_off = b;
  b = align_up(b + sizeof(Tile) * L.tiles.size(), kAlign);
  L.ptiles_off = b;
  b = align_up(b + sizeof(Tile) * L.ptiles.size(), kAlign);
  // TMA descriptors of the staged mixed step: [copy][domain]
  L.tmaps_off = b;
  if (c->storage != RLBM_F64) b = align_up(b + 2 * (size_t)kTensorMapBytes * L.dd.size(), kAlign);
  L.pop_off[0] = b;
  b += L.pop_bytes;
  L.pop_off[1] = b;
  b += L.pop_bytes;
  L.total = b;
}

}  // namespace

struct rlbm_ctx {
  int edf = 0, storage = 0, ndom = 0;
  std::vector<rlbm_domain> doms;
  Layout L;
  char* base = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  unsigned* d_status = nullptr;
  DomDev* d_doms = nullptr;
  Tile* d_tiles = nullptr;
  Tile* d_ptiles = nullptr;          // the packed tile list (Layout::ptiles)
  unsigned char* d_tmaps = nullptr;  // null unless the TMA-staged variant is available
  void* pop[2] = {nullptr, nullptr};
  int cur = 0;
  std::vector<char> initialized;
  cudaGraphExec_t pair_graph[2] = {nullptr, nullptr};
  cudaGraphExec_t chunk_graph[2] = {nullptr, nullptr};
  unsigned* h_status = nullptr;  // pinned
  long long last_updates = 0;
  int last_launches = 0;
  long long cells = 0;
  int grid = 0;                  // blocks of the step kernel (0 = one per tile)
  int kernel = RLBM_KERNEL_L1;   // mixed step variant (rlbm_select_kernel)
  unsigned long long wait_ns = 0;  // TMA copy-wait limit (0: the default, rlbm_set_wait_limit)
  bool images_stale = false;     // the current copy lacks its periodic halo images (fill_images)
  int halo = 2;                  // halo work of a step launch (StepArgs::halo)
};

namespace {

int cuda_fail(cudaError_t e) { return e == cudaSuccess ? RLBM_OK : RLBM_E_CUDA; }

// The tile list a step launch walks: the packed one for the mixed step's L1
// pull, the plain one for the TMA-staged variant (whose boxes assume 32 x
// kTileH tiles) and the FP64 step.
bool packed_tiles(const rlbm_ctx* h) { return h->storage != RLBM_F64 && h->kernel == RLBM_KERNEL_L1; }

cudaError_t launch_step(rlbm_ctx* h, int from) {
  StepArgs a;
  a.doms = h->d_doms;
  const bool pk = packed_tiles(h);
  a.tiles = pk ? h->d_ptiles : h->d_tiles;
  a.ntiles = (int)(pk ? h->L.ptiles.size() : h->L.tiles.size());
  a.fin = h->pop[from];
  a.fout = h->pop[1 - from];
  a.status = h->d_status;
  // descriptors [copy][domain]: the loads of copy `from`
  const size_t per = (size_t)h->ndom * kTensorMapBytes;
  const bool tma = h->d_tmaps && h->kernel == RLBM_KERNEL_TMA;
  a.tmaps = tma ? h->d_tmaps + (size_t)from * per : nullptr;
  a.variant = h->kernel;
  a.wait_ns = h->wait_ns;
  a.halo = h->halo;
  const int grid = h->grid > 0 ? h->grid : a.ntiles;
  if (h->storage == RLBM_F64) return launch_step_f64(h->edf, a, grid, h->stream);
  return launch_step_mixed(h->storage, h->edf, a, grid, h->stream);
}

// Capture `nsteps` (even) steps starting from copy `from` into an executable graph.
cudaError_t capture(rlbm_ctx* h, int from, int nsteps, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaSuccess;
  int c = from;
  for (int i = 0; i < nsteps; ++i) {
    cudaError_t r = launch_step(h, c);
    if (r != cudaSuccess && le == cudaSuccess) le = r;
    c = 1 - c;
  }
  e = cudaStreamEndCapture(h->stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

// TMA descriptors of the staged mixed step, written into `out` as
// [copy][domain]: a 4D tensor {32 lanes, 72 planes, nblk blocks, ny + 2 rows}
// of the copy's elements (the halo ring included), boxes {32, 6, 3, kTileH + 2} (one
// direction's six shell planes, the tile's block and its neighbours, rows
// y0-1 .. y0+kTileH), zero fill outside. Returns false if the driver offers no
// encoder or refuses a descriptor; the handle then has only the L1 variant.
bool encode_tmaps(const rlbm_ctx* h, std::vector<unsigned char>& out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();  // clear the non-sticky error the failed query recorded
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const size_t es = h->L.esize;
  const size_t nd = (size_t)h->ndom;
  out.assign(2 * (size_t)kTensorMapBytes * nd, 0);
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  for (int copy = 0; copy < 2; ++copy)
    for (size_t i = 0; i < nd; ++i) {
      const DomDev& D = h->L.dd[i];
      char* base = static_cast<char*>(h->pop[copy]) + (size_t)D.off * es;  // 256-byte aligned
      const cuuint64_t dims[4] = {(cuuint64_t)kBlkW, (cuuint64_t)kNq, (cuuint64_t)D.nblk, (cuuint64_t)D.ny + 2};
      const cuuint64_t strides[3] = {(cuuint64_t)kBlkW * es, (cuuint64_t)kBlk * es, (cuuint64_t)D.pitch * es};
      const cuuint32_t box[4] = {(cuuint32_t)kBlkW, (cuuint32_t)kBoxPlanes, (cuuint32_t)kBoxBlocks,
                                 (cuuint32_t)kBoxRows};
      CUtensorMap* m = reinterpret_cast<CUtensorMap*>(out.data() + ((size_t)copy * nd + i) * kTensorMapBytes);
      if (encode(m, dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    }
  return true;
}

// Forget the captured step graphs (they bake in the launch configuration).
void drop_graphs(rlbm_ctx* h) {
  for (int i = 0; i < 2; ++i) {
    if (h->pair_graph[i]) cudaGraphExecDestroy(h->pair_graph[i]);
    if (h->chunk_graph[i]) cudaGraphExecDestroy(h->chunk_graph[i]);
    h->pair_graph[i] = h->chunk_graph[i] = nullptr;
  }
}

// Staging area for host transfers: the population copy that does not hold the
// current state (it is overwritten by the next step anyway).
double* staging(rlbm_ctx* h) { return static_cast<double*>(h->pop[1 - h->cur]); }
size_t staging_doubles(rlbm_ctx* h) { return h->L.pop_bytes / sizeof(double); }

constexpr int kSlabPlanes = 30;  // 5 directions with v_y of one sign x 6 shells
constexpr int kPlanesUp = 6;     // q = 6..35: d = 1..5, v_y > 0
constexpr int kPlanesDown = 42;  // q = 42..71: d = 7..11, v_y < 0

// One domain's rows in a population copy.
struct RowArgs {
  DomDev D;         // geometry (nx, ny, nblk, pitch, off)
  int unpack;       // 0: edge rows -> packed faces, 1: packed faces -> ghost rows
  void* pop;
  void* face[2];    // low, high; either may be null
};

// Raw element copy between a packed [30][nx + 2] face and one row of 30
// planes, both faces in one launch (the storage encoding is kept as is).
template <class T>
__global__ void k_rows(RowArgs a) {
  const long long w = a.D.nx + 2, per = kSlabPlanes * w;
  T* pop = static_cast<T*>(a.pop);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 2 * per;
       e += (long long)gridDim.x * blockDim.x) {
    const int side = e >= per;
    T* buf = static_cast<T*>(a.face[side]);
    if (!buf) continue;
    const long long r = e - side * per, k = r / w, xx = r % w;
    // sent rows: row 0 down (planes 42..), row ny-1 up (planes 6..);
    // received rows: y = -1 gets planes 6.., y = ny gets planes 42..
    const int q0 = (side == 0) == (a.unpack != 0) ? kPlanesUp : kPlanesDown;
    const int y = a.unpack ? (side ? a.D.ny : -1) : (side ? a.D.ny - 1 : 0);
    int x = (int)xx - 1;
    // a sent row's periodic x ghosts are its wrapped end cells (the L1 step
    // leaves the images unwritten)
    if (!a.unpack && a.D.bc[0] == BC_PERIODIC) x = x < 0 ? a.D.nx - 1 : (x == a.D.nx ? 0 : x);
    const long long idx = cell_pos(a.D, x, y) + (q0 + k) * kBlkW;
    if (a.unpack) pop[idx] = buf[r];
    else buf[r] = pop[idx];
  }
}

// Periodic halo images of every domain of a population copy, copied from the
// interior cells they map to (raw elements, all 72 planes): pass 0 the x
// images of rows -1..ny, then pass 1 the y images of columns -1..nx (so the
// corners take the images of the x ghosts). The result is the halo the
// producing step would have written with its images on.
template <class T>
__global__ void k_images(const DomDev* doms, int ndom, void* pop_, int pass) {
  T* pop = static_cast<T*>(pop_);
  for (int dm = blockIdx.y; dm < ndom; dm += gridDim.y) {
    const DomDev& D = doms[dm];
    if (D.bc[pass == 0 ? 0 : 2] != BC_PERIODIC) continue;
    const long long len = pass == 0 ? D.ny + 2 : D.nx + 2, per = 72 * len;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 2 * per;
         e += (long long)gridDim.x * blockDim.x) {
      const int side = e >= per;
      const long long r = e - side * per;
      const int q = (int)(r / len), k = (int)(r % len) - 1;
      long long dst, src;
      if (pass == 0) {
        dst = cell_pos(D, side ? D.nx : -1, k);
        src = cell_pos(D, side ? 0 : D.nx - 1, k);
      } else {
        dst = cell_pos(D, k, side ? D.ny : -1);
        src = cell_pos(D, k, side ? 0 : D.ny - 1);
      }
      pop[dst + q * kBlkW] = pop[src + q * kBlkW];
    }
  }
}

cudaError_t fill_images(rlbm_ctx* h) {
  if (!h->images_stale) return cudaSuccess;
  const dim3 grid(64, (unsigned)std::min(h->ndom, 65535));
  for (int pass = 0; pass < 2; ++pass) {
    switch (h->L.esize) {
      case 8: k_images<unsigned long long><<<grid, 256, 0, h->stream>>>(h->d_doms, h->ndom, h->pop[h->cur], pass); break;
      case 4: k_images<unsigned><<<grid, 256, 0, h->stream>>>(h->d_doms, h->ndom, h->pop[h->cur], pass); break;
      default: k_images<unsigned short><<<grid, 256, 0, h->stream>>>(h->d_doms, h->ndom, h->pop[h->cur], pass); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  h->images_stale = false;
  return cudaSuccess;
}

int slab_rows(rlbm_handle h, int domain, void* lo, void* hi, int unpack) {
  if (!h || domain < 0 || domain >= h->ndom) return RLBM_E_ARG;
  if (!h->initialized[domain]) return RLBM_E_STATE;
  const size_t es = h->L.esize;
  if ((reinterpret_cast<uintptr_t>(lo) % es) || (reinterpret_cast<uintptr_t>(hi) % es)) return RLBM_E_ARG;
  if (!lo && !hi) return RLBM_OK;
  const DomDev& D = h->L.dd[domain];
  RowArgs a;
  a.D = D;
  a.unpack = unpack;
  a.pop = h->pop[h->cur];
  a.face[0] = lo;
  a.face[1] = hi;
  const long long n = 2LL * kSlabPlanes * (D.nx + 2);
  // one element per thread, at most 8 blocks of 256 per SM (152 SMs); the loop strides beyond
  const int grid = (int)std::min<long long>((n + 255) / 256, 8 * 152);
  switch (es) {
    case 8: k_rows<unsigned long long><<<grid, 256, 0, h->stream>>>(a); break;
    case 4: k_rows<unsigned><<<grid, 256, 0, h->stream>>>(a); break;
    default: k_rows<unsigned short><<<grid, 256, 0, h->stream>>>(a); break;
  }
  return cuda_fail(cudaGetLastError());
}

}  // namespace

extern "C" {

size_t rlbm_workspace_bytes(const rlbm_config* c) {
  if (validate(c)) return 0;
  Layout L;
  make_layout(c, L);
  return L.total;
}

int rlbm_layout_tiles(const rlbm_config* c, int packed, int* out, int max_tiles) {
  if (validate(c) || max_tiles < 0) return RLBM_E_ARG;
  Layout L;
  make_layout(c, L);
  const std::vector<Tile>& t = packed ? L.ptiles : L.tiles;
  if (out)
    for (size_t i = 0; i < t.size() && (long long)i < max_tiles; ++i) {
      out[4 * i + 0] = t[i].dom;
      out[4 * i + 1] = t[i].x0;
      out[4 * i + 2] = t[i].y0;
      out[4 * i + 3] = t[i].w;
    }
  return (int)t.size();
}

int rlbm_create(const rlbm_config* c, rlbm_handle* out) {
  if (!out) return RLBM_E_ARG;
  *out = nullptr;
  int v = validate(c);
  if (v) return v;
  rlbm_ctx* h = new (std::nothrow) rlbm_ctx();
  if (!h) return RLBM_E_ARG;
  h->edf = c->edf;
  h->storage = c->storage;
  h->ndom = c->ndomains;
  h->doms.assign(c->domains, c->domains + c->ndomains);
  make_layout(c, h->L);
  if (!c->device_buffer || c->buffer_bytes < h->L.total ||
      (reinterpret_cast<uintptr_t>(c->device_buffer) % kAlign)) {
    delete h;
    return RLBM_E_NOBUFFER;
  }
  h->halo = 0;
  for (const rlbm_domain& d : h->doms) {
    h->cells += (long long)d.nx * d.ny;
    for (int b : {d.bc_xlo, d.bc_xhi, d.bc_ylo, d.bc_yhi})
      if (bc_writes_halo(b)) h->halo = std::max(h->halo, b == RLBM_FIXED_T_WALL ? 1 : 2);
  }
  h->base = static_cast<char*>(c->device_buffer);
  h->d_status = reinterpret_cast<unsigned*>(h->base + h->L.status_off);
  h->d_doms = reinterpret_cast<DomDev*>(h->base + h->L.doms_off);
  h->d_tiles = reinterpret_cast<Tile*>(h->base + h->L.tiles_off);
  h->d_ptiles = reinterpret_cast<Tile*>(h->base + h->L.ptiles_off);
  if (h->storage != RLBM_F64) h->d_tmaps = reinterpret_cast<unsigned char*>(h->base + h->L.tmaps_off);
  h->pop[0] = h->base + h->L.pop_off[0];
  h->pop[1] = h->base + h->L.pop_off[1];
  h->initialized.assign(h->ndom, 0);
  cudaError_t e = cudaSuccess;
  if (c->cuda_stream) {
    h->stream = static_cast<cudaStream_t>(c->cuda_stream);
  } else {
    e = cudaStreamCreate(&h->stream);  // blocking w.r.t. the legacy default stream
    h->own_stream = true;
  }
  if (e == cudaSuccess) e = prepare_f64();
  if (e == cudaSuccess) e = prepare_mixed();
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_status, sizeof(unsigned));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_doms, h->L.dd.data(), sizeof(DomDev) * h->L.dd.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_tiles, h->L.tiles.data(), sizeof(Tile) * h->L.tiles.size(),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_ptiles, h->L.ptiles.data(), sizeof(Tile) * h->L.ptiles.size(),
                        cudaMemcpyHostToDevice, h->stream);
  std::vector<unsigned char> maps;
  if (e == cudaSuccess && h->d_tmaps && !encode_tmaps(h, maps)) h->d_tmaps = nullptr;
  if (e == cudaSuccess && h->d_tmaps)
    e = cudaMemcpyAsync(h->d_tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = launch_prepare_refs(h->edf, h->d_doms, h->ndom, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    rlbm_destroy(h);
    return RLBM_E_CUDA;
  }
  *out = h;
  return RLBM_OK;
}

int rlbm_init(rlbm_handle h, int domain, int kind, const double* a, const double* theta,
              const double* ux, const double* uy, int on_device) {
  if (!h || domain < 0 || domain >= h->ndom || !a || !theta || !ux || !uy) return RLBM_E_ARG;
  if (kind != RLBM_INIT_N_THETA && kind != RLBM_INIT_Z_THETA) return RLBM_E_ARG;
  const rlbm_domain& d = h->doms[domain];
  const size_t n = (size_t)d.nx * d.ny;
  const double *da = a, *dt = theta, *dx = ux, *dy = uy;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    if (4 * n > staging_doubles(h)) return RLBM_E_UNSUPPORTED;
    double* s = staging(h);
    e = cudaMemcpyAsync(s, a, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s + n, theta, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s + 2 * n, ux, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s + 3 * n, uy, n * 8, cudaMemcpyHostToDevice, h->stream);
    da = s; dt = s + n; dx = s + 2 * n; dy = s + 3 * n;
  }
  if (e != cudaSuccess) return RLBM_E_CUDA;
  // status of this call only
  unsigned saved = 0;
  e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  saved = *h->h_status;
  e = cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream);
  InitArgs ia;
  ia.doms = h->d_doms;
  ia.dom = domain;
  ia.kind = kind;
  ia.a = da; ia.theta = dt; ia.ux = dx; ia.uy = dy;
  ia.f = h->pop[h->cur];
  ia.status = h->d_status;
  ia.tiles = nullptr;
  ia.ntiles = 0;
  if (e == cudaSuccess)
    e = h->storage == RLBM_F64 ? launch_init_f64(h->edf, ia, d.nx, d.ny, h->stream)
                               : launch_init_mixed(h->storage, h->edf, ia, d.nx, d.ny, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  const unsigned st = *h->h_status;
  // restore earlier step warnings so rlbm_sync_status still reports them
  *h->h_status = saved;
  e = cudaMemcpyAsync(h->d_status, h->h_status, sizeof(unsigned), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  h->initialized[domain] = 1;
  return (int)st;
}

int rlbm_step(rlbm_handle h, int nsteps) {
  if (!h || nsteps < 0) return RLBM_E_ARG;
  for (char v : h->initialized)
    if (!v) return RLBM_E_STATE;
  int launches = 0;
  // the TMA-staged step reads the periodic halo images as stored
  cudaError_t e = h->storage != RLBM_F64 && h->kernel == RLBM_KERNEL_TMA && nsteps > 0 ? fill_images(h)
                                                                                        : cudaSuccess;
  int left = nsteps;
  while (left >= 2 * kChunkPairs && e == cudaSuccess) {
    if (!h->chunk_graph[h->cur]) e = capture(h, h->cur, 2 * kChunkPairs, &h->chunk_graph[h->cur]);
    if (e == cudaSuccess) e = cudaGraphLaunch(h->chunk_graph[h->cur], h->stream);
    left -= 2 * kChunkPairs;
    launches += 2 * kChunkPairs;
  }
  while (left >= 2 && e == cudaSuccess) {
    if (!h->pair_graph[h->cur]) e = capture(h, h->cur, 2, &h->pair_graph[h->cur]);
    if (e == cudaSuccess) e = cudaGraphLaunch(h->pair_graph[h->cur], h->stream);
    left -= 2;
    launches += 2;
  }
  if (left == 1 && e == cudaSuccess) {
    e = launch_step(h, h->cur);
    h->cur = 1 - h->cur;
    launches += 1;
  }
  if (nsteps > 0 && packed_tiles(h)) h->images_stale = true;  // the L1 step wraps instead
  h->last_updates = (long long)nsteps * h->cells;
  h->last_launches = launches;
  return cuda_fail(e);
}

int rlbm_moments(rlbm_handle h, int domain, int streamed, double* n, double* theta, double* ux,
                 double* uy, double* z, int on_device) {
  if (!h || domain < 0 || domain >= h->ndom || !n || !theta || !ux || !uy) return RLBM_E_ARG;
  if (!h->initialized[domain]) return RLBM_E_STATE;
  const rlbm_domain& d = h->doms[domain];
  const size_t cnt = (size_t)d.nx * d.ny;
  FieldsArgs fa;
  fa.diag = nullptr;
  fa.tiles = nullptr;
  fa.ntiles = 0;
  fa.doms = h->d_doms;
  fa.dom = domain;
  fa.streamed = streamed ? 1 : 0;
  fa.f = h->pop[h->cur];
  fa.status = h->d_status;
  if (on_device) {
    fa.n = n; fa.theta = theta; fa.ux = ux; fa.uy = uy; fa.z = z;
  } else {
    if (5 * cnt > staging_doubles(h)) return RLBM_E_UNSUPPORTED;
    double* s = staging(h);
    fa.n = s; fa.theta = s + cnt; fa.ux = s + 2 * cnt; fa.uy = s + 3 * cnt; fa.z = s + 4 * cnt;
  }
  cudaError_t e = h->storage == RLBM_F64 ? launch_fields_f64(h->edf, fa, d.nx, d.ny, h->stream)
                                          : launch_fields_mixed(h->storage, h->edf, fa, d.nx, d.ny, h->stream);
  if (e == cudaSuccess && !on_device) {
    double* outs[5] = {n, theta, ux, uy, z};
    double* srcs[5] = {fa.n, fa.theta, fa.ux, fa.uy, fa.z};
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
      if (outs[k]) e = cudaMemcpyAsync(outs[k], srcs[k], cnt * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  return cuda_fail(e);
}

int rlbm_init_all(rlbm_handle h, int kind, const double* a, const double* theta, const double* ux,
                  const double* uy, int on_device) {
  if (!h || !a || !theta || !ux || !uy) return RLBM_E_ARG;
  if (kind != RLBM_INIT_N_THETA && kind != RLBM_INIT_Z_THETA) return RLBM_E_ARG;
  const size_t n = (size_t)h->cells;
  const double *da = a, *dt = theta, *dx = ux, *dy = uy;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    if (4 * n > staging_doubles(h)) return RLBM_E_UNSUPPORTED;
    double* s = staging(h);
    e = cudaMemcpyAsync(s, a, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s + n, theta, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s + 2 * n, ux, n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s + 3 * n, uy, n * 8, cudaMemcpyHostToDevice, h->stream);
    da = s; dt = s + n; dx = s + 2 * n; dy = s + 3 * n;
  }
  if (e != cudaSuccess) return RLBM_E_CUDA;
  // this call's status only: read and keep the earlier bits, clear, launch,
  // read this call's bits, put the earlier ones back
  e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  const unsigned saved = *h->h_status;
  e = cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream);
  InitArgs ia;
  ia.doms = h->d_doms;
  ia.dom = 0;
  ia.kind = kind;
  ia.a = da; ia.theta = dt; ia.ux = dx; ia.uy = dy;
  ia.f = h->pop[h->cur];
  ia.status = h->d_status;
  ia.tiles = h->d_tiles;
  ia.ntiles = (int)h->L.tiles.size();
  if (e == cudaSuccess)
    e = h->storage == RLBM_F64 ? launch_init_f64(h->edf, ia, 0, 0, h->stream)
                               : launch_init_mixed(h->storage, h->edf, ia, 0, 0, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  const unsigned st = *h->h_status;
  *h->h_status = saved;
  e = cudaMemcpyAsync(h->d_status, h->h_status, sizeof(unsigned), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  for (char& v : h->initialized) v = 1;
  h->images_stale = false;  // the initialisers write the periodic images too
  return (int)st;
}

int rlbm_moments_all(rlbm_handle h, int streamed, double* n, double* theta, double* ux, double* uy, double* z,
                     int on_device) {
  if (!h || !n || !theta || !ux || !uy) return RLBM_E_ARG;
  for (char v : h->initialized)
    if (!v) return RLBM_E_STATE;
  const size_t cnt = (size_t)h->cells;
  FieldsArgs fa;
  fa.diag = nullptr;
  fa.tiles = h->d_tiles;
  fa.ntiles = (int)h->L.tiles.size();
  fa.doms = h->d_doms;
  fa.dom = 0;
  fa.streamed = streamed ? 1 : 0;
  fa.f = h->pop[h->cur];
  fa.status = h->d_status;
  if (on_device) {
    fa.n = n; fa.theta = theta; fa.ux = ux; fa.uy = uy; fa.z = z;
  } else {
    if (5 * cnt > staging_doubles(h)) return RLBM_E_UNSUPPORTED;
    double* s = staging(h);
    fa.n = s; fa.theta = s + cnt; fa.ux = s + 2 * cnt; fa.uy = s + 3 * cnt; fa.z = s + 4 * cnt;
  }
  cudaError_t e = h->storage == RLBM_F64 ? launch_fields_f64(h->edf, fa, 0, 0, h->stream)
                                          : launch_fields_mixed(h->storage, h->edf, fa, 0, 0, h->stream);
  if (e == cudaSuccess && !on_device) {
    double* outs[5] = {n, theta, ux, uy, z};
    double* srcs[5] = {fa.n, fa.theta, fa.ux, fa.uy, fa.z};
    for (int k = 0; k < 5 && e == cudaSuccess; ++k)
      if (outs[k]) e = cudaMemcpyAsync(outs[k], srcs[k], cnt * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  return cuda_fail(e);
}

int rlbm_diagnostics(rlbm_handle h, int domain, int streamed, double* out, int on_device) {
  if (!h || domain < 0 || domain >= h->ndom || !out) return RLBM_E_ARG;
  if (!h->initialized[domain]) return RLBM_E_STATE;
  const rlbm_domain& d = h->doms[domain];
  const size_t cnt = (size_t)d.nx * d.ny;
  FieldsArgs fa;
  fa.tiles = nullptr;
  fa.ntiles = 0;
  fa.doms = h->d_doms;
  fa.dom = domain;
  fa.streamed = streamed ? 1 : 0;
  fa.f = h->pop[h->cur];
  fa.status = h->d_status;
  fa.n = fa.theta = fa.ux = fa.uy = fa.z = nullptr;
  if (on_device) {
    fa.diag = out;
  } else {
    if (7 * cnt > staging_doubles(h)) return RLBM_E_UNSUPPORTED;
    fa.diag = staging(h);
  }
  cudaError_t e = h->storage == RLBM_F64 ? launch_fields_f64(h->edf, fa, d.nx, d.ny, h->stream)
                                          : launch_fields_mixed(h->storage, h->edf, fa, d.nx, d.ny, h->stream);
  if (e == cudaSuccess && !on_device) {
    e = cudaMemcpyAsync(out, fa.diag, 7 * cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  return cuda_fail(e);
}

static int copy_pops(rlbm_handle h, int domain, double* f, int on_device, int to_dense) {
  if (!h || domain < 0 || domain >= h->ndom || !f) return RLBM_E_ARG;
  const rlbm_domain& d = h->doms[domain];
  const size_t per_plane = (size_t)(d.nx + 2) * (d.ny + 2);
  CopyArgs ca;
  ca.doms = h->d_doms;
  ca.dom = domain;
  ca.to_dense = to_dense;
  ca.pop = h->pop[h->cur];
  auto launch = [&](const CopyArgs& a) {
    return h->storage == RLBM_F64 ? launch_copy_f64(a, h->stream) : launch_copy_mixed(h->storage, a, h->stream);
  };
  cudaError_t e = cudaSuccess;
  if (on_device) {
    ca.q0 = 0;
    ca.nq = 72;
    ca.dense = f;
    e = launch(ca);
  } else {
    // stage through the spare population copy, as many planes at a time as fit
    const int chunk = (int)std::min<size_t>(72, staging_doubles(h) / per_plane);
    if (chunk < 1) return RLBM_E_UNSUPPORTED;
    for (int q0 = 0; q0 < 72 && e == cudaSuccess; q0 += chunk) {
      ca.q0 = q0;
      ca.nq = std::min(chunk, 72 - q0);
      ca.dense = staging(h);
      const size_t bytes = (size_t)ca.nq * per_plane * sizeof(double);
      double* host = f + (size_t)q0 * per_plane;
      if (!to_dense) e = cudaMemcpyAsync(ca.dense, host, bytes, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = launch(ca);
      if (e == cudaSuccess && to_dense) e = cudaMemcpyAsync(host, ca.dense, bytes, cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
  }
  if (e == cudaSuccess && !to_dense) h->initialized[domain] = 1;
  return cuda_fail(e);
}

int rlbm_get_populations(rlbm_handle h, int domain, double* f, int on_device) {
  if (h && domain >= 0 && domain < h->ndom && !h->initialized[domain]) return RLBM_E_STATE;
  if (h && fill_images(h) != cudaSuccess) return RLBM_E_CUDA;  // a checkpoint holds the whole halo
  return copy_pops(h, domain, f, on_device, 1);
}

int rlbm_set_populations(rlbm_handle h, int domain, const double* f, int on_device) {
  return copy_pops(h, domain, const_cast<double*>(f), on_device, 0);
}

size_t rlbm_edge_row_bytes(rlbm_handle h, int domain) {
  if (!h || domain < 0 || domain >= h->ndom) return 0;
  return (size_t)kSlabPlanes * (size_t)(h->doms[domain].nx + 2) * h->L.esize;
}

int rlbm_pack_edge_rows(rlbm_handle h, int domain, void* lo, void* hi) {
  return slab_rows(h, domain, lo, hi, 0);
}

int rlbm_unpack_ghost_rows(rlbm_handle h, int domain, const void* lo, const void* hi) {
  return slab_rows(h, domain, const_cast<void*>(lo), const_cast<void*>(hi), 1);
}

int rlbm_tune(rlbm_handle h, int repeats) {
  if (!h || repeats < 1) return RLBM_E_ARG;
  for (char v : h->initialized)
    if (!v) return RLBM_E_STATE;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  // grid 0: one block per tile of whichever list the variant walks
  const int ntiles = (int)h->L.ptiles.size();  // the shorter list
  std::vector<int> cand = {0};
  for (int k : {1, 2, 3, 4, 6, 8})
    if (k * sms < ntiles) cand.push_back(k * sms);
  // keep the warnings accumulated so far; timing launches must not add any
  e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  const unsigned saved = *h->h_status;
  cudaEvent_t t0, t1;
  if (cudaEventCreate(&t0) != cudaSuccess) return RLBM_E_CUDA;
  if (cudaEventCreate(&t1) != cudaSuccess) { cudaEventDestroy(t0); return RLBM_E_CUDA; }
  // kernel variants: the mixed storages with TMA descriptors have two
  std::vector<int> kernels = {RLBM_KERNEL_L1};
  if (h->d_tmaps) kernels.push_back(RLBM_KERNEL_TMA);
  if (h->d_tmaps && fill_images(h) != cudaSuccess) {  // the TMA candidates time on the stored halo
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return RLBM_E_CUDA;
  }
  float best = 1e30f;
  int best_grid = 0, best_kernel = h->kernel;
  for (int kv : kernels)
    for (int g : cand) {
      h->kernel = kv;
      h->grid = g;
      e = launch_step(h, h->cur);  // reads the current copy, writes the spare one
      if (e == cudaSuccess) e = cudaEventRecord(t0, h->stream);
      for (int r = 0; r < repeats && e == cudaSuccess; ++r) e = launch_step(h, h->cur);
      if (e == cudaSuccess) e = cudaEventRecord(t1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      if (e != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        best_grid = g;
        best_kernel = kv;
      }
    }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  h->grid = best_grid;
  h->kernel = best_kernel;
  if (best_grid == 0) best_grid = (int)(packed_tiles(h) ? h->L.ptiles.size() : h->L.tiles.size());
  drop_graphs(h);
  *h->h_status = saved;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_status, h->h_status, sizeof(unsigned), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? best_grid : RLBM_E_CUDA;
}

int rlbm_set_grid(rlbm_handle h, int grid) {
  if (!h || grid < 0) return RLBM_E_ARG;
  if (grid != h->grid) {
    h->grid = grid;
    drop_graphs(h);  // the captured launches hold the old grid
  }
  return grid;
}

int rlbm_select_kernel(rlbm_handle h, int kernel) {
  if (!h) return RLBM_E_ARG;
  if (kernel < 0) return h->kernel;
  if (kernel != RLBM_KERNEL_L1 && kernel != RLBM_KERNEL_TMA) return RLBM_E_ARG;
  if (kernel == RLBM_KERNEL_TMA && !h->d_tmaps) return RLBM_E_UNSUPPORTED;
  if (kernel != h->kernel) {
    h->kernel = kernel;
    drop_graphs(h);
  }
  return kernel;
}

int rlbm_set_wait_limit(rlbm_handle h, double seconds) {
  if (!h || seconds != seconds) return RLBM_E_ARG;
  unsigned long long ns = 0;  // the default
  if (seconds > 0.0) ns = seconds >= 1e9 ? ~0ull >> 1 : std::max(1ull, (unsigned long long)(seconds * 1e9));
  if (ns != h->wait_ns) {
    h->wait_ns = ns;
    drop_graphs(h);  // the captured launches hold the old limit
  }
  return RLBM_OK;
}

int rlbm_sync_status(rlbm_handle h) {
  if (!h) return RLBM_E_ARG;
  cudaError_t e = cudaMemcpyAsync(h->h_status, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return RLBM_E_CUDA;
  return (int)*h->h_status;
}

int rlbm_destroy(rlbm_handle h) {
  if (!h) return RLBM_E_ARG;
  for (int i = 0; i < 2; ++i) {
    if (h->pair_graph[i]) cudaGraphExecDestroy(h->pair_graph[i]);
    if (h->chunk_graph[i]) cudaGraphExecDestroy(h->chunk_graph[i]);
  }
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->h_status) cudaFreeHost(h->h_status);
  delete h;
  return RLBM_OK;
}

const char* rlbm_status_string(int code) {
  switch (code) {
    case RLBM_OK: return "ok";
    case RLBM_E_ARG: return "invalid argument";
    case RLBM_E_CUDA: return "a CUDA call failed";
    case RLBM_E_STATE: return "call out of order (initialise every domain first)";
    case RLBM_E_UNSUPPORTED: return "unsupported combination";
    case RLBM_E_NOBUFFER: return "device workspace missing, misaligned or too small";
    case RLBM_E_SCRATCH: return "domain too large for the fixed scratch of rlbm_step_noalloc";
    default: break;
  }
  if (code > 0) {
    if (code & RLBM_W_DEVICE_TIMEOUT) return "error: a bounded device wait timed out (step results invalid)";
    if (code & RLBM_W_NONPHYSICAL) return "warning: non-physical state in some cell (left unrelaxed)";
    if (code & RLBM_W_ZSOLVE) return "warning: fugacity solve did not converge in some cell";
    if (code & RLBM_W_LANDAU_MAXITER) return "warning: Landau solve hit its iteration cap";
    if (code & RLBM_W_CLAMPED_FUGACITY) return "warning: BE fugacity clamped to z_c";
  }
  return "unknown status";
}

int rlbm_last_step_info(rlbm_handle h, long long* cell_updates, int* kernel_launches) {
  if (!h) return RLBM_E_ARG;
  if (cell_updates) *cell_updates = h->last_updates;
  if (kernel_launches) *kernel_launches = h->last_launches;
  return RLBM_OK;
}

}  // extern "C"
