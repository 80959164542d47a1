// plan.h -- work descriptors shared by the host planner and the leaf-GEMM kernels.
//
// A launch of the grouped leaf GEMM processes a list of LEAVES.  A leaf is one sub-product
// P = Aop * Bop of the recursion (Sec. 2.2 / 2.3) whose operands are rectangles of tensor
// maps (the input matrices or the materialised operand sums), and whose result is added with
// a sign into one or more TARGET blocks of C -- the post-additions U1..U7 (or C11..C22 of
// Strassen) folded into the epilogue.  A leaf is cut into BM x BN output tiles; every tile is
// one work item of the persistent kernel.
#pragma once
#include <cstdint>

namespace swk {

// Device error word values (the host maps them to SW_ETIMEOUT / SW_ECUDA).
enum : int {
    ERR_NONE = 0,
    ERR_WAIT_FULL = 1,      // MMA waited too long for a TMA stage
    ERR_WAIT_EMPTY = 2,     // producer waited too long for a free stage
    ERR_WAIT_ACC = 3,       // epilogue waited too long for an accumulator
    ERR_WAIT_ACC_FREE = 4,  // MMA waited too long for the epilogue to free an accumulator
    ERR_WAIT_DRAIN = 5,     // final drain of in-flight copies / MMAs
    ERR_ALIGN = 6,          // a TMA coordinate violated the 16-byte rule (the copy was skipped)
    ERR_ORDER = 7,          // an ordered epilogue waited too long for its predecessor
    ERR_UNITS = 9,          // a launch with an explicit work layout got another number of units
};

// With ordering counters (flag_base >= 0), the STORE of a tile is the block's first write: its
// epilogue warps each add 1 to the tile's counter once their stores are complete, and every
// ATOMIC contribution to the same tile waits until the counter reaches 4 * epoch first.
enum TargetMode : int {
    TGT_STORE = 0,   // C_block  = sign * P
    TGT_ATOMIC = 1,  // C_block += sign * P  (atomic; several leaves may hit the block at once)
    TGT_ADD = 2,     // C_block += sign * P  (plain read-modify-write; single writer at a time)
};

struct Target {
    void* c;          // origin of the target block (element type of the product)
    long long ldc;    // leading dimension in elements
    int rows, cols;   // valid extent of the block; rows/cols beyond it are not written
    float sign;       // +1 or -1
    int mode;         // TargetMode
    int vec_ok;       // 1 when c is 16-byte aligned and ldc is a multiple of 4 (FP32)
    int map;          // index of the block's tensor map for TMA store / reduce-add (-1: none)
    int flag_base;    // ordering counters of this block's tiles (-1: unordered)
    int flag_cols;    // tiles per row of the block (counter index = tile_row * flag_cols + tile_col)
};

struct Leaf {
    int a_map, b_map;  // tensor-map indices
    int a_row, a_col;  // origin of the A operand in its map (row, column)
    int b_row, b_col;  // origin of the B operand in its map; for the TF32 kernel the map holds
                       // B^T, so b_row indexes N and b_col indexes K
    int m, n;          // extent of the product (tiles_m = ceil(m/BM), tiles_n = ceil(n/BN))
    int kblocks;       // number of BK-deep k blocks
    int tgt_begin, tgt_count;
    int tile_begin;    // index of the leaf's first work item
    int tiles_n;
    int c_row0, c_col0;  // position of the leaf's tile (0, 0) inside its target blocks
    int tag;             // resident server: completion counter of the leaf's request (-1: none)
    int cont;            // 1: the tile continues the accumulator of this CTA's last tile that used
                         //    the same TMEM accumulator (two items back with two accumulators, the
                         //    previous item with one); an accumulation chain, which needs an
                         //    explicit item table (see ResidentCtl)
    int a_job, b_job;    // launches that pack operands themselves (ResidentCtl::pack_jobs): the
                         // jobs writing this leaf's A / B, whose tiles must be complete before its
                         // loads (-1: none); read by no other launch
};

struct CopyJob;

// Work source of the resident (serving) form of the grouped GEMM: items are published by the
// host while the kernel runs.  `published` and `stop` live in host-mapped memory; each CTA claims
// published items one at a time (compare-and-swap on `next`) and, after `idle_ns` without new
// work, exits.  Every epilogue warp adds 1 to done[leaf.tag] when its part of a tile is stored.
struct ResidentCtl {
    unsigned* next;                   // device: next unclaimed item
    const volatile unsigned* published;  // host-mapped: items the host has published
    const volatile unsigned* stop;       // host-mapped: nonzero asks the kernel to exit
    const int* item_leaf;             // device: leaf index of every published item
    unsigned* done;                   // device: per-request completion counters
    unsigned long long idle_ns;
    // Non-resident launches may carry an explicit work layout: item_tile[i] = tile row << 16 | tile
    // column of item i (with item_leaf[i] its leaf), planned for exactly `units` persistent units
    // (CTAs, or CTA pairs) so that unit u processes items u, u + units, ... in order.
    const int* item_tile;
    int units;
    // Non-resident batched launches may also pack operands: extra warps copy the tiles of
    // pack_jobs (CopyJob::pad_ = the job's tile count) and count each finished tile on the job's
    // ordering counter, which a leaf's producer waits for (Leaf::a_job / b_job).
    const CopyJob* pack_jobs;
    int pack_njobs, pack_tiles;
};

}  // namespace swk
