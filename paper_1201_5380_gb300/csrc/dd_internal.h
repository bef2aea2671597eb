// Internal declarations of the GB300 dedispersion library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dedisp.h"

namespace dd {

// ---------------------------------------------------------------------------
// Staged image ("lane format").  Before dedispersion the time-major input is
// turned into one row per channel, samples packed along time into 32-bit
// words: word w of a row holds image samples [w*SPW, (w+1)*SPW), sample i
// of the word in lane i (bits [i*LW, (i+1)*LW)).  Image sample s is time
// s - kPad: a left pad keeps every staging window start non-negative.
// Lane widths leave guard bits above the data so that several channels can
// be added lane-parallel (the bit-level parallelism of Sec. 2.3):
//   FMT_NIB  4-bit lanes, 8 samples/word, 1- and 2-bit input
//   FMT_BYTE 8-bit lanes, 4 samples/word, 4-bit input
//   FMT_HALF 16-bit lanes, 2 samples/word, 8-bit input and sub-band stage 2
//   FMT_U32  32-bit unsigned, 1 sample/word, wide sub-band intermediates
//   FMT_F32  32-bit float, 1 sample/word, float input
//   FMT_TRI  10-bit lanes at bits [0,10), [10,20), [20,30), 3 samples/word,
//            8-bit input of the direct transform (4 channels fit a lane)
//   FMT_SB8  8-bit lanes, 4 samples/word: sub-band stage 2 over stage-1
//            sums below 128 (1- and 2-bit input), two sub-bands a lane
// ---------------------------------------------------------------------------
enum Fmt {
  FMT_NIB = 0, FMT_BYTE = 1, FMT_HALF = 2, FMT_U32 = 3, FMT_F32 = 4, FMT_TRI = 5, FMT_SB8 = 6
};
// OUT_NARROW: scaled uint8/uint16 rows (LaunchParams::out_bits, out_shift),
// a separate instantiation so the uint32 kernel's code is untouched.
// OUT_HALFIMG / OUT_BYTEIMG: sub-band stage-1 rows written as the stage-2
// image, in 16-bit (FMT_HALF) or 8-bit (FMT_SB8) lanes.
enum OutKind { OUT_U32 = 0, OUT_F32 = 1, OUT_HALFIMG = 2, OUT_NARROW = 3, OUT_BYTEIMG = 4 };

constexpr int kPad = 32;  // image samples before time 0 (multiple of 4*SPW)

inline int fmt_spw(int fmt) {
  switch (fmt) {
    case FMT_NIB: return 8;
    case FMT_BYTE: return 4;
    case FMT_SB8: return 4;
    case FMT_HALF: return 2;
    case FMT_TRI: return 3;
    default: return 1;
  }
}

// Device status flags (OR-ed by kernels, read by dd_plan_get_device_status).
enum : uint32_t {
  DEV_BAD_WINDOW = 1u,  // a lane window ran past the staged copy
  DEV_BAD_READ = 2u,    // staging read past an image row
  DEV_BAD_ITEM = 4u,    // malformed work item
  DEV_TIMEOUT = 8u,     // a bounded wait for a bulk copy expired
};

// One regular grid of work: n_groups groups, each `ndm` trials (`ndm_last` in
// the last group) x nsamps outputs over one image.  Group g uses the image,
// delay table and output advanced by g times the group strides (sub-bands in
// sub-band stage 1, trial groups in stage 2; a direct job has one group).
// Items of a segment are (tile group, group, trial block), trial block
// fastest; a tile group is tiles_per_item consecutive time tiles, which one
// item stages and sums as one stream of chunks.
struct Seg {
  const int32_t* blk;     // optional trial-block starts (n_dmblk + 1 entries,
                          // device); null = regular blocks of B trials
  const uint32_t* img;    // image row of channel 0 (group 0)
  const int32_t* delays;  // delay of trial 0, channel 0 (group 0)
  void* out;              // output row of trial 0 at time 0 (group 0)
  int64_t row_words;      // image row pitch, words
  int64_t out_stride;     // output row pitch (elements; words for the image outputs)
  int64_t nsamps;         // outputs per trial
  int64_t item_begin;     // first global item index of this segment
  int64_t tile0;          // first time tile of the segment's first item
  int64_t tile_end;       // the segment's items cover tiles [tile0, tile_end)
  int64_t g_img;          // per-group image offset, words
  int64_t g_out;          // per-group output offset, elements (words)
  int32_t g_delay;        // per-group delay-table offset, elements
  int32_t n_groups;       // >= 1
  int32_t ndm;            // trials per group
  int32_t ndm_last;       // trials in the last group
  int32_t n_dmblk;        // ceil(ndm / trials per block)
  int32_t delay_stride;   // elements between trial rows of the delay table
  int32_t nchan;          // channels summed
  int32_t tiles_per_item; // time tiles per item (>= 1)
  int32_t lo_slack;       // max_{block,c} delay(d0,c) - min_{d in block} delay(d,c)
  // Staging tables of the launch geometry (built on the host, see StageTab):
  const uint32_t* atab;   // [group][block: atab_blk][chunk][trial slot][channel
                          // of chunk] byte offset of the (trial, channel) window
  const int32_t* crec;    // per group, pairs: [block][channel] {window start word
                          // - t0/SPW, words of the window the block's trials
                          // read}, then [block] the block's chunk geometry
                          // {channels per chunk, window words}
  int64_t g_atab;         // per-group offsets of the two tables (elements)
  int64_t g_crec;
  int64_t atab_blk;       // atab entries per block (channels rounded up to the
                          // largest chunk, x trial slots)
};

constexpr int kMaxSegs = 32;  // segments per launch, passed inline as a kernel parameter

struct LaunchParams {
  Seg segs[kMaxSegs];
  int32_t n_segs;
  // chunk geometry: per trial block from its staging tables (per_block_geo),
  // else every block of the launch stages cc channels in windows of nww words
  int32_t per_block_geo;
  int32_t cc, nww;
  int32_t f0, f1, f2;  // flush periods (groups of 4 channels) per level
  int64_t n_items;
  uint32_t* status;
  // work-item counter (zeroed before the launch): blocks take their next
  // item from it, so the blocks running at any moment work on neighbouring
  // items (and share the staged windows of a tile in L2) however long the
  // launch; null = static striding by the grid size
  unsigned long long* next_item;
  int32_t vec_out;   // 1 if every output row/tile start is 16-byte aligned
  int32_t out_bits;  // 32, or 16 / 8: scaled output (OUT_U32 launches)
  int32_t out_shift; // scaled output = min(sum >> out_shift, 2^out_bits - 1)
  int32_t multi_tile; // 1 if any segment's items cover several tiles (MT kernel)
};

// The plan's status buffer: the status word, then kItemCounters launch
// counters taken round-robin, so launches of one plan that overlap on
// different streams do not share a counter.
constexpr int kItemCounters = 32;
constexpr size_t kStatusBytes = 8 + 8 * kItemCounters;

// Kernel shapes compiled into the library.
struct TileCfg {
  int nwarp, dpw, k;  // warps per block, trials per warp, words per lane
};
// (16, 2, 8) is for the narrow-accumulator formats (4-bit and wider input,
// where a wide window over a short tile makes staging dominate); the
// 4-bit-lane format compiles it too but spills, as do the 8-bit lanes with
// 32-bit accumulators.  (16, 2, 16) is compiled only
// for the one- and two-sample-a-word formats (16-bit lanes, 32-bit words),
// whose accumulators take one or two registers a word: short work items
// (the sub-band method's second stage) gain most from its longer tiles.
constexpr TileCfg kTileCfgs[] = {{16, 2, 4}, {16, 4, 2}, {8, 2, 4}, {8, 4, 2}, {16, 2, 8},
                                 {16, 2, 16}};
constexpr int kNumTileCfgs = 6;

// Host launchers (dd_kernels_*.cu).
cudaError_t launch_dedisp(int fmt, int outk, bool wide, int cfg, const LaunchParams& p,
                          int grid, size_t smem, cudaStream_t st);
cudaError_t dedisp_max_blocks_per_sm(int fmt, int outk, bool wide, int cfg, bool pbg, bool mt,
                                     size_t smem, int* nblk);
// Whether the multi-tile kernel (items of several time tiles) is compiled
// for this staged format, output kind, accumulator width and tile shape.
bool multi_tile_compiled(int fmt, int outk, bool wide, int cfg);
// Whether only the multi-tile kernel is compiled for them (the 8-bit-lane
// sub-band stages): their launches always take it, one tile an item or more.
bool multi_tile_only(int fmt, int outk);
// Image words [w_first, words) of every channel row, in staged format fmt
// (fmt_for_nbits, or FMT_HALF for 8-bit input of the sub-band method).
cudaError_t launch_corner_turn(int nbits, int fmt, const uint8_t* in, int64_t in_stride,
                               int64_t t_begin, int64_t nrows_valid, int nchans,
                               const uint8_t* mask, uint32_t* img, int64_t row_words,
                               int64_t w_first, int64_t words, cudaStream_t st);

size_t dedisp_smem_bytes(int fmt, int cfg, int cc, int nww);
cudaError_t launch_probe(const uint32_t* seed, int64_t iters, uint32_t* sink, int grid,
                         cudaStream_t st);

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf();
  cudaError_t ensure(size_t n);  // grow-only
  void release();
};

struct Tuning {
  int dms_per_block = 32;
  int chans_per_chunk = 32;  // the most; each trial block's own fits its windows
  int words_per_lane = 0;  // 0: chosen per input format (tuning_for)
};

// Staging tables of one delay table for one launch geometry.  They do not
// depend on the time tile: a tile starts on a multiple of 4*SPW samples, so
// each (trial block, channel) window starts at t0/SPW + woff image words and
// every trial's offset inside it is fixed.
struct StageTab {
  bool uploaded = false;
  std::vector<uint32_t> atab;  // see Seg::atab
  std::vector<int32_t> crec;   // see Seg::crec (pairs)
  int64_t g_atab = 0, g_crec = 0, atab_blk = 0;
  size_t smem = 0;             // dynamic shared memory of the widest block
  bool uniform = false;        // every block has chunk geometry (cc, nww)
  int cc = 0, nww = 0;
  int64_t reach = 0;           // image words past t0/SPW that any tile's windows read
  DevBuf d_atab, d_crec;
};

// Where a stage table's delays come from (host copies).
struct TabSrc {
  const int32_t* delays;  // group 0, trial 0, channel 0
  int64_t g_delay;        // per-group offset (elements)
  int dstride;            // elements between trial rows
  int nchan, ngroups;
  const int32_t* blk;     // per-group block starts, nblk+1 entries per group
  int nblk;
  int lo;                 // lo_slack of the blocks
};

struct Plan {
  int device = 0;
  int nchans = 0;
  double dt = 0, f0 = 0, df = 0;
  std::vector<double> dms;
  std::vector<int32_t> delays;  // ndm x nchans
  std::vector<uint8_t> mask;    // nchans
  int32_t max_delay = 0;
  int64_t gulp = 0;
  int sb_chans = 0, sb_dms = 0;  // sub-band N', N'_DM (0 = off)
  bool sb_centred = false;       // nominal trial: group's middle (else lowest)
  Tuning tune;
  bool tuned_by_search = false;
  int num_sms = 0;

  // device state
  DevBuf d_delays, d_mask, d_status, d_image, d_in, d_out;
  DevBuf d_sb_rel, d_sb_d2, d_sb_S;
  bool delays_dirty = true, mask_dirty = true, sb_dirty = true, sb_dev_dirty = true;
  std::vector<int32_t> sb_rel, sb_d2;  // host copies of the sub-band tables
  int32_t sb_max_delay = 0;
  int64_t sb_len1_extra = 0;  // max_{d,n} delay(d, nN')
  // staging spreads (incl. lo_slack) and lo_slack per trials-per-block
  // B = 16 << i, for the direct table and the two sub-band stages
  int32_t spread_B[3] = {0, 0, 0}, lo_B[3] = {0, 0, 0};
  std::vector<int32_t> blocks_B[3];  // trial-block starts (+ end) per B
  DevBuf d_blk[3];
  bool blk_dirty = true;
  int32_t sb1_spread_B[3] = {0, 0, 0}, sb1_lo_B[3] = {0, 0, 0};
  int32_t sb2_spread_B[3] = {0, 0, 0}, sb2_lo_B[3] = {0, 0, 0};
  int32_t sb_maxrel = 0;
  // per-group trial-block tables of the two sub-band stages, per B
  std::vector<int32_t> sb1_blk_B[3], sb2_blk_B[3];
  int32_t sb1_nblk_B[3] = {0, 0, 0}, sb2_nblk_B[3] = {0, 0, 0};
  DevBuf d_sb1_blk[3], d_sb2_blk[3];
  // staging tables: key {kind (0 direct, 1/2 sub-band stage), tile shape,
  // format, chunk cap, lo_slack, window width, blocks}.  An entry is never
  // rebuilt in place (a launch on another stream may still read it).  The
  // cache is bounded: entries go when the delays change or when it is full
  // and a launch needs a new uploaded table.  They are shared: a captured
  // graph keeps the tables its kernels read alive however the cache changes.
  std::map<std::array<int, 7>, std::shared_ptr<StageTab>> tabs;
  // kernel timing (dd_plan_set_kernel_timing)
  bool timing = false;
  struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<TimedLaunch> timed;
  double timed_ms[3] = {0.0, 0.0, 0.0};  // per kind (DD_KERNEL_*)
  int64_t timed_n[3] = {0, 0, 0};
  // time-scrunching (Sec. 2.2): 0 = off, else the largest factor; trials at
  // one factor form a level, run by a child plan at resolution s*dt
  int out_bits = 32;  // bits per output sample of dd_execute (8, 16 or 32)
  int scrunch_max = 0;
  bool scr_dirty = true;
  struct ScrLevel {
    int s, d_lo, d_hi;
    std::unique_ptr<Plan> plan;
  };
  std::vector<ScrLevel> scr_levels;
  std::vector<int32_t> scr_factor;  // per trial
  DevBuf d_scr;                     // scrunched input of the level being run
  // piecewise linear tree (Sec. 3.1.1): N' channels per sub-band (0 = off)
  int tree_chans = 0;
  bool tree_dirty = true, tree_dev_dirty = true;
  std::vector<int32_t> tree_tab;   // [trial][sub-band] {stage-1 row, shift}
  std::vector<int32_t> tree_roff;  // first stage-1 row of each sub-band (+ end)
  int32_t tree_shift_max = 0;      // max_{d,n} dt''_n(d)
  DevBuf d_tree_tab, d_tree_roff, d_tree_S;
  // host-pointer execute: output copies overlap the next part's compute
  cudaStream_t copy_st = nullptr;  // host-output path: copies out
  cudaStream_t in_st = nullptr;    // host-output path: input rows in
  std::vector<cudaEvent_t> part_ev;
  uint32_t launch_seq = 0;  // round-robin index into the item counters
  std::mutex mu;
  ~Plan();
};

// Bracket a kernel launch with events when the plan's timing is enabled.
struct KernelTimer {
  Plan* p;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  KernelTimer(Plan* plan, int k, cudaStream_t s);
  ~KernelTimer();
};

inline int b_index(int B) { return B <= 16 ? 0 : (B <= 32 ? 1 : 2); }

int ndm(const Plan& p);
dd_status ensure_device_tables(Plan& p);
dd_status prepare_subband(Plan& p);  // host tables only
dd_status upload_subband(Plan& p);   // host tables + device copies
int tile_cfg_index(const Tuning& t);
bool have_tile_cfg(int dms_per_block, int words_per_lane);  // a compiled shape
// The tuning a launch of staged format fmt uses: words per lane 0 resolves
// to 8 for the narrow-accumulator formats (16- and 32-bit lanes: 8-bit and
// float input, the sub-band intermediate) and 4 otherwise, when a compiled
// tile shape has that many trials per block and words per lane.
Tuning tuning_for(const Tuning& t, int fmt);

// Direct and sub-band execution on device buffers (asynchronous on st).
struct ExecArgs {
  int64_t nsamps_out;
  const void* in;
  int in_nbits;
  int64_t in_row_stride;
  int64_t in_rows;      // rows available in `in` (>= nsamps_out + max_delay)
  void* out;
  int64_t out_stride;
  cudaStream_t st;
  bool subband;
  bool tree = false;  // piecewise linear tree (Sec. 3.1.1)
};
dd_status exec_device(Plan& p, const ExecArgs& a);
// Time-scrunched direct transform (device pointers); input rows needed.
dd_status exec_scrunch(Plan& p, const ExecArgs& a);
dd_status prepare_scrunch(Plan& p);
int64_t scrunch_input_rows(const Plan& p, int64_t nsamps_out);
dd_status build_delays(Plan& p);
// Eq. 3: samples of delay per unit DM of channel c (any c >= 0 whose
// frequency is positive, including the band edge c = nchans).
double partial_delay(double f0, double df, double dt, int c);
// Piecewise linear tree (Sec. 3.1.1): host tables, input rows beyond the
// gulp, and the two-stage execution on device buffers.
dd_status prepare_tree(Plan& p);
int64_t tree_input_extra(const Plan& p);
dd_status exec_tree(Plan& p, const ExecArgs& a);
void plan_init_band(Plan& p, int nchans, double dt, double f0, double df);

// Build the segments and launch parameters for a direct transform over an
// already staged image (used by execute, streams and batches).
struct DirectJob {
  const uint32_t* img;
  int64_t row_words;
  int64_t img_row_samples;  // valid image samples per row incl. left pad
  const int32_t* d_delays;  // device delay table (ndm x nchans)
  const int32_t* h_delays;  // host copy (planning)
  int nchans;
  int ndm;
  int64_t nsamps;
  void* out;
  int64_t out_stride;
  const Plan* plan;  // owner of the delay table (cached staging spreads)
  const int32_t* blk_dev = nullptr;  // device block table; null = the plan's own
  bool no_upload = false;  // leave staging tables on the host (caller places them)
};

struct LaunchPlan {
  int fmt, outk, cfg;
  bool wide;
  LaunchParams lp;
  std::vector<Seg> segs;
  size_t smem;
  int grid;
};

// Image geometry for a job of nsamps outputs with max delay maxd.
int64_t image_row_words(int fmt, const Tuning& t, int64_t nsamps, int32_t maxd,
                        int32_t spread);
int32_t max_block_spread(const int32_t* delays, int ndm, int nchans, int stride,
                         int B, int32_t* lo_slack);
// Cut trials into blocks of at most B whose staging spread stays within
// budget samples (a lone trial always forms a block); returns the block
// starts plus the end, and the largest spread / lo_slack of the blocks.
void make_blocks(const int32_t* delays, int ndm, int nchans, int stride, int B,
                 int32_t budget, std::vector<int32_t>* starts, int32_t* spread,
                 int32_t* lo_slack);
// Largest staging spread (samples) of a trial block: with double-buffered
// staging and 4-channel chunks the windows of every format then fit in
// 220 KB of shared memory.
constexpr int32_t kSpreadBudget = 4000;
// Dynamic shared memory a dedispersion block may use for its staging buffers.
constexpr size_t kSmemCap = 220 * 1024;
int time_tile(int fmt, const Tuning& t);
int out_elem_bytes(const Plan& p, int outk);
bool out_vec_ok(const void* out, int64_t stride_elems, int esz);
dd_status plan_direct_launch(Plan& p, int fmt, int outk, int vmax,
                             const std::vector<DirectJob>& jobs, LaunchPlan* lpl,
                             std::vector<std::shared_ptr<StageTab>>* tabs = nullptr);
// timer_kind: the DD_KERNEL_* kind the launch is timed under
dd_status run_launch(Plan& p, LaunchPlan& lpl, cudaStream_t st, int timer_kind = 1);
// The plan's staging tables of `src` (kind 0 direct, 1/2 sub-band stage)
// for a launch geometry, built on first use and uploaded when asked; null
// with *err set if a window would not fit the geometry.  Without upload
// nothing is allocated or freed on the device: a table not yet cached is
// cached only while the cache has room, else returned to the caller alone.
std::shared_ptr<StageTab> stage_tab(Plan& p, int kind, const TabSrc& src, int fmt, int cfg,
                                    int cc_cap, int nww_uniform, bool upload, dd_status* err);
void drop_stage_tabs(Plan& p, int kind_mask);
dd_status stage_direct_image(Plan& p, const void* in, int nbits, int64_t in_stride, int64_t rows,
                             int64_t nsamps, DevBuf& image, cudaStream_t st, DirectJob* j);

dd_status cuda_status(cudaError_t e);
// Staged format of the direct transform for nbits input over nchans
// channels (-1: unsupported nbits).  8-bit input takes 10-bit lanes, three
// samples a word, while a lane's whole sum fits 20 bits (nchans * 255 <
// 2^20, up to 4112 channels), else 16-bit lanes.
int fmt_for_nbits(int nbits, int nchans);
int vmax_for_nbits(int nbits);

}  // namespace dd
