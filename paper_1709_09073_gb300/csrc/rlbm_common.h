// Definitions shared by the host side of the C ABI and the CUDA kernels.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace rlbm {

enum { EDF_MJ = 0, EDF_FD = 1, EDF_BE = 2 };
enum { BC_PERIODIC = 0, BC_ZERO_GRADIENT = 1, BC_WALL = 2, BC_VWALL = 3, BC_EXCHANGED = 4 };
// a side whose ghost is an equilibrium (fixed-T or velocity wall)
__host__ __device__ inline bool bc_is_wall(int b) { return b == BC_WALL || b == BC_VWALL; }
// a side whose ghost the step writes (not periodic: the pull wraps; not
// exchanged: the caller supplies it)
__host__ __device__ inline bool bc_writes_halo(int b) { return b != BC_PERIODIC && b != BC_EXCHANGED; }
enum { ST_F64 = 0, ST_F32 = 1, ST_BF16DEV = 2, ST_F16DEV = 3, ST_F32DEV = 4 };

// per-cell status bits (identical to the public RLBM_W_* values)
enum { ST_LANDAU = 1, ST_CLAMPED = 2, ST_NONPHYSICAL = 4, ST_ZSOLVE = 8, ST_TIMEOUT = 16 };

constexpr double PI = 3.14159265358979323846264338327950288;
constexpr double ZC = 1.0 - 1.0e-7;  // BE reference fugacity, Eq. (15)
constexpr double SQRT3_2 = 0.86602540378443864676372317075294;

// Population layout: blocks of 32 cells of a row, each block holding all 72
// populations of its cells ("array of structures of arrays"): element (q, x, y),
// x in [-1, nx], y in [-1, ny] (the halo ring included), lives at
//   off + (y + 1) * pitch + ((x + 32) / 32) * kBlk + q * kBlkW + (x + 32) % 32,
// so a warp's access to one population of 32 cells is one aligned 32-element
// segment, the 72 segments of a block are contiguous, and the offset of plane
// q is the constant q * kBlkW. Block 0 of a row holds x = -32 .. -1 (only x = -1
// is used); pitch = nblk * kBlk with nblk = (nx + 32) / 32 + 1 blocks per row.
constexpr int kBlkW = 32;           // cells per x block
constexpr int kNq = 72;             // populations per cell
constexpr int kBlk = kNq * kBlkW;   // elements per x block

struct DomDev {
  int nx, ny, nblk, pad0;
  long long pitch;        // elements per row of blocks (nblk * kBlk)
  long long off;          // element offset of the domain within a population copy
  long long foff;         // offset of the domain's cells in packed [sum ny*nx] field arrays
  int bc[4];              // xlo, xhi, ylo, yhi
  int order, pad_;        // expansion order N of Eq. (10), 2..5
  double inv_tau;
  double t_wall[4];
  double ref_n, ref_theta;  // reference rest equilibrium (deviation form of the mixed path)
  double scale;             // deviation scale of the 16-bit storage
  double eta_s;             // > 0: local tau = 4 eta_s / theta + 0.2546 (Sec. 3.5); else inv_tau
  double tau;               // constant relaxation time (inv_tau = 1 / tau)
  double accel_x, accel_y;  // body acceleration: the collision uses u + a tau (Sec. 3.4)
  double n_wall;            // density of the velocity-wall sides
  // filled on the device from (ref_n, ref_theta) at handle creation:
  double zref[6];           // isotropic equilibrium moments Z_n0 of the reference state
  double n0ref, t00ref;     // N^0 and T^00 of the FP32 reference populations fref
  double zeff1, zeff2;      // n0ref, t00ref plus the N^0, T^00 of the residual rres
  float n0_hl[2], t00_hl[2], z1_hl[2], z2_hl[2];  // the same four as double-float pairs
  float zref_f[6];          // zref rounded to FP32
  float fref[6];            // reference populations per shell (FP32)
  float rres[6];            // FP64 reference equilibrium minus fref, per shell
  float a_s[6];             // 16-bit storage: f = fref + a_s * h, a_s = fref * scale
  float b_s[6];             // 1 / a_s
  float inv_tau_f, eta_s_f;  // inv_tau and eta_s rounded to FP32 (the mixed step issues no FP64)
  float t_wall_f[4];         // t_wall rounded to FP32
};

// Cells of one work-list tile along x and y. Every step kernel covers one tile
// per block and is launched with blocks of kTileW x kTileH threads; the host
// builds the tile lists (rlbm_create, rlbm_step_noalloc) from the same
// constants. kTileW is one x block of the population layout.
#ifndef RLBM_TILE_H
#define RLBM_TILE_H 4
#endif
constexpr int kTileW = 32, kTileH = RLBM_TILE_H;

// A tile of domain `dom` from cell (x0, y0). w = 0: kTileW x kTileH cells, warp
// k on row y0 + k, lane l on x0 + l. w in 1..kPackMaxW: the ragged last x
// block of a domain, only w cells wide, packed: each warp covers 32 / w rows of
// w cells (lane l on x0 + l % w, row y0 + k * (32 / w) + l / w; lanes from
// (32 / w) * w on idle), so the tile spans kTileH * (32 / w) rows.
struct Tile {
  int dom, x0, y0, w;
};
constexpr int kPackMaxW = 16;  // widest ragged block worth packing (two rows per warp)

__host__ __device__ constexpr int packed_rows_per_warp(int w) { return w > 0 ? kTileW / w : 1; }

// Cell of thread (lane, warp) of a tile; false for idle lanes of a packed tile
// (cells outside the domain are the caller's test).
__host__ __device__ inline bool tile_cell(const Tile& tl, int lane, int warp, int& x, int& y) {
  if (tl.w == 0) {
    x = tl.x0 + lane;
    y = tl.y0 + warp;
    return true;
  }
  const int r = kTileW / tl.w;
  x = tl.x0 + lane % tl.w;
  y = tl.y0 + warp * r + lane / tl.w;
  return lane < r * tl.w;
}

struct StepArgs {
  const DomDev* doms;
  const Tile* tiles;
  int ntiles;
  const void* fin;        // population copy read (post-collision, with halo)
  void* fout;             // population copy written
  unsigned* status;       // OR of per-cell status bits
  const void* tmaps;      // TMA load descriptors of fin, one per domain (kTensorMapBytes each), or null
  int variant;            // mixed step kernel (RLBM_KERNEL_*); the FP64 step has one
  int halo;               // halo work of the launch: 0 none (every side periodic or exchanged),
                          // 1 wall equilibria only, 2 also zero-gradient copies
  unsigned long long wait_ns;  // limit of the TMA variant's copy waits (0: kDefaultWaitNs)
};

constexpr unsigned long long kDefaultWaitNs = 1000000000ull;  // one second

// Element index of cell (x, y), plane 0 (add q * kBlkW for plane q), from the
// start of the domain (cell_rel) or of the population copy (cell_pos).
__host__ __device__ inline long long cell_rel(const DomDev& D, int x, int y) {
  const int X = x + kBlkW;  // >= 31
  return (long long)(y + 1) * D.pitch + (long long)(X / kBlkW) * kBlk + (X % kBlkW);
}
__host__ __device__ inline long long cell_pos(const DomDev& D, int x, int y) { return D.off + cell_rel(D, x, y); }

// Blocks of 32 cells per row for a domain nx cells wide (halo blocks included).
__host__ __device__ constexpr int blocks_per_row(int nx) { return (nx + kBlkW) / kBlkW + 1; }

constexpr int kTensorMapBytes = 128;  // sizeof(CUtensorMap), 64-byte aligned in memory

// TMA box of the staged mixed step: for one direction, the six shell planes of
// the tile's x block and its two neighbours over rows y0-1 .. y0+kTileH, i.e. a
// box {32 lanes, 6 planes, 3 blocks, kTileH + 2 rows} of the 4D tensor
// {32 lanes, 72 planes, nblk blocks, ny + 2 rows}.
constexpr int kBoxRows = kTileH + 2, kBoxBlocks = 3, kBoxPlanes = 6;
constexpr int kBoxElems = kBlkW * kBoxPlanes * kBoxBlocks * kBoxRows;

}  // namespace rlbm
