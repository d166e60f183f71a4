// wave_shape.h -- launch-shape limits of the band wavefront (K2), shared by
// the kernel (launch bounds) and the host (shape checks, planner).
#pragma once

namespace dfd {
namespace wave {

constexpr int G = 32;        // systolic steps between synchronisations
constexpr int RING = 256;    // columns held by each inter-warp ring (power of 2)

// q columns per TMA chunk.  A compute warp checks a chunk's barrier once per
// chunk, and the warp that paces the band pays a few hundred cycles for it:
// 512-column chunks (8 slots: a ring of 4096 columns, about 138 KB of
// shared memory for 3-D points) made the 200,000^2 pair 2.5% faster than
// 128-column ones (16 slots).
constexpr int chunk_cols(int dk) { return dk <= 4 ? 512 : 128; }

// q chunk slots (a power of 2).  Points of up to 4 coordinates keep 4 slots
// of 512 columns (about 70 KB of shared memory a CTA for 3-D points), so two
// CTAs fit an SM and each SM sub-partition holds two compute warps (one
// compute warp per sub-partition left the step's dependent chain exposed);
// larger points keep 8 slots of 128 columns and one CTA per SM.
constexpr int nq_slots(int C) { return C >= 512 ? 4 : 8; }
// CTAs an SM can hold at the planner's shapes (the occupancy query decides
// at launch; the kernel is compiled for one CTA per SM, so a CTA may also
// have as many warps as the register file allows).
constexpr int blocks_per_sm(int dk) { return dk <= 4 ? 2 : 1; }

// Column skew between neighbouring lanes: float32 lanes hold R/2 skewed row
// pairs, int32 lanes keep their R rows in one column.
constexpr int skew(bool f32, int R) { return f32 ? R / 2 : 1; }

// Deadlock bound of the q ring.  Warp w+1 needs columns that warp w emits
// 32*K - 1 columns late and publishes per G-block, so it trails warp w by at
// most 32*K + G columns; lane 31 of the last warp reads 31*K columns behind
// its lane 0, and warp 0 waits for the chunks one block ahead (the q
// look-ahead reaches two columns past the block).  Every chunk warp 0 can
// wait for must fit in the ring beside the oldest one the last warp may
// still read:
//   (NQ - 1) * C >= (W - 1) * (32*K + G) + 31*K + G + 2.
constexpr int max_warps_ring(int C, int K) { return ((nq_slots(C) - 1) * C - 31 * K - G - 2) / (32 * K + G) + 1; }

// Registers a compute lane needs (points, row state, q records in flight,
// the block's ring inputs, addressing), an estimate calibrated on ptxas.
// The narrow int32 class (uint32 bits carried as floats) runs the float32
// stripe with integer coordinates and one |p|^2 more per row.
constexpr int reg_estimate(bool f32, int dk, int R, bool narrow = false) {
  return f32 ? 48 + R * dk + (R / 2) * ((dk + 1) / 2) * 4 + 2 * R + 3 * (R / 2) + G + (narrow ? R : 0)
             : 48 + R * dk + 4 * R + ((dk + 3) / 4) * 4;
}

// Compute warps per CTA the register file allows (with the communication
// warp, one CTA per SM); 0 if even one warp would not fit in 255 registers.
constexpr int max_warps_regs(bool f32, int dk, int R, bool narrow = false) {
  return reg_estimate(f32, dk, R, narrow) > 248 ? 0
         : (65536 / (32 * ((reg_estimate(f32, dk, R, narrow) + 7) / 8 * 8)) - 1) > 16
             ? 16
             : 65536 / (32 * ((reg_estimate(f32, dk, R, narrow) + 7) / 8 * 8)) - 1;
}

constexpr bool shape_supported(bool f32, int dk, int R, int W) {
  return (R == 2 || R == 4 || R == 6 || R == 8) && W >= 1 && W <= max_warps_regs(f32, dk, R) &&
         W <= max_warps_ring(chunk_cols(dk), skew(f32, R));
}

// An int32 pair launches both its kernels with one shape: the narrow one
// (float32 stripe and skew) and the exact int64 one.
constexpr bool narrow_shape_supported(int dk, int R, int W) {
  return (R == 2 || R == 4 || R == 6 || R == 8) && W >= 1 && W <= max_warps_regs(true, dk, R, true) &&
         W <= max_warps_ring(chunk_cols(dk), skew(true, R));
}
constexpr bool int_shape_supported(int dk, int R, int W) {
  return shape_supported(false, dk, R, W) && narrow_shape_supported(dk, R, W);
}

}  // namespace wave
}  // namespace dfd
