// g6gb_internal.h -- declarations shared by the kernels and the C-ABI layer
// of the GRAPE-6-style force library (arXiv:0902.4463).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "g6gb.h"

namespace g6 {

// j-particles per shared-memory tile and padding unit of j-memory.  The
// force kernels stream j in tiles of this size; j-memory is padded to a
// multiple of it with massless particles far away (Sect. 2.3, Fig. accMP:
// each thread block stages j-particles in shared memory and loops over them).
constexpr int JT = 256;

// An i-tile whose work is spread over at most this many CTAs is reduced by
// the last of them inside the force launch; more partials go to K3, whose
// many CTAs beat the serial tail of one.
constexpr int FUSED_MAX_SEGS = 4;

// One partial result of a (work segment, i-particle) pair: sums over the
// j-range the segment covers (Sect. 2.3: partial forces of the P blocks are
// reduced on the GPU before the copy back).
//
// DS path: each sum as a compensated FP32 pair (hi, lo), about 48 bits; the
// reductions stay in compensated FP32 and convert to FP64 once per result,
// because GB300's FP64 pipe is about 1/64 of its FP32 rate.  64 bytes.
struct PartialDS {
    float2 acc[3], jerk[3], pot;  // pot accumulates +m/r; negated at the end
    float nnr2;                   // smallest unsoftened |r|^2 seen
    int nnj;                      // its j-slot, -1 if none
};
// All-FP64 path: plain FP64 sums.  72 bytes.
struct Partial64 {
    double acc[3], jerk[3], pot;
    double nnr2;
    int nnj;
    int pad;
};
// Bytes of one partial slot whichever path writes it.
constexpr size_t PARTIAL_BYTES = sizeof(Partial64) > sizeof(PartialDS) ? sizeof(Partial64)
                                                                         : sizeof(PartialDS);
using Partial = Partial64;   // slot-sized unit of partial buffers

// One tile of JT j-slots of the raw j-store as one contiguous block, so that
// a kernel stages a tile with one bulk copy (one stream per tile keeps HBM at
// full rate; one stream per array would halve it): the planes, each JT
// entries and 16-byte aligned, are t0 (double), (v, m), a/2, j/6 (float4),
// (x_hi, y_hi, z_hi, x_lo) (float4), (y_lo, z_lo) (float2), index (int) --
// 84 B per slot, 21504 B per tile.
constexpr unsigned RAW_T0 = 0;
constexpr unsigned RAW_V = RAW_T0 + JT * 8;
constexpr unsigned RAW_A = RAW_V + JT * 16;
constexpr unsigned RAW_J = RAW_A + JT * 16;
constexpr unsigned RAW_XA = RAW_J + JT * 16;
constexpr unsigned RAW_XB = RAW_XA + JT * 16;
constexpr unsigned RAW_ID = RAW_XB + JT * 8;
constexpr unsigned RAW_TILE_BYTES = RAW_ID + JT * 4;

// j-memory (the j-store), capacity `cap` (multiple of JT).
struct JStore {
    double *x0;        // 3 planes of cap doubles: x, y, z at t0 (FP64)
    unsigned char *raw;    // cap / JT tiles in the layout above: t0, FP32 copies of
                           // (v, m), a/2, j/6, the position as double-single, index
    double4_32a *v64;      // (vx, vy, vz, m)              FP64 copy
    double4_32a *a264;     // (ax/2, ay/2, az/2, 0)
    double4_32a *j664;     // (jx/6, jy/6, jz/6, 0)
    int *idx;          // particle index (-1: empty slot), flat: the same values as
                       // the tiles' index plane, for the reductions and the FP64 path
    int cap;
};

// Words per j-particle of the predicted DS layout and their order inside a
// tile: each tile of JT j-particles is one contiguous block of JW * JT
// 32-bit words, component-major (all x_hi of the tile, then all y_hi, ...),
// so that one bulk copy stages a tile and a thread reads two consecutive
// j-particles of one component as a float2.
constexpr int JW = 11;
enum JWord { W_XH = 0, W_YH, W_ZH, W_M, W_XL, W_YL, W_ZL, W_VX, W_VY, W_VZ, W_ID };

// Predicted j-particles (force-kernel input).
struct Pred {
    float *pt;         // DS: tiled layout above, cap / JT tiles
    int2 *trange;      // DS: per tile, smallest and largest particle index
                       //     (empty tile: INT_MAX, -1); lets the force kernel
                       //     skip the per-pair self test on tiles that hold
                       //     none of its i-particles
    double4_32a *p64;      // FP64: (x, y, z, m)
    double4_32a *v64;      // FP64: (vx, vy, vz, index)
};

// A force launch: kernel variant, CTA shape and the work partition.  The
// work line is n_itile * J (i-tile, j-tile) pairs cut into `grid` equal
// contiguous ranges, one per CTA (Sect. 2.3: j split over the
// multiprocessors, i split into segments, j split again for small blocks).
struct ForceConfig {
    int variant;       // index into the variant table
    int ti, tj, nper;  // threads along i, along j, i-particles per thread
    int itile;         // ti * nper
    int grid;          // CTAs
    int jtiles;        // J
    int n_itile;
    long long work;    // n_itile * J
    int smem;          // dynamic shared memory bytes
    int list;          // builds neighbour lists
    int prec;          // G6X_PREC_*
    int ws;            // warp-specialised small-block kernel (launch_force_ws)
};

// Shape of one compiled force-kernel variant.
struct VariantInfo {
    int ti, tj, nper, list, prec;
    int fpred = 0;     // predicts the j-tiles itself (Eq. 1, Eq. 2) from the raw j-store
    int twin = -1;     // for fpred shapes: the same shape reading predicted tiles
    int ws = 0;        // warp-specialised small-block kernel: the whole block is one
                       // i-tile, j-tiles streamed by a producer warp, the partials
                       // reduced inside the launch (two levels)
};

// What a fused-prediction force kernel needs: the raw j-store, the block
// time and the number of particles in j-memory (DS + SP predictor only).
struct FusedPred {
    JStore js;
    double t;
    int nj;
    // staged j-records sorted by tile (toff: per-tile ranges), stored by
    // the force kernel itself; only with one i-tile (NULL: none staged)
    const g6x_jrec *rec = nullptr;
    const int *toff = nullptr;
};

// Work geometry of a batch of independent clusters: cluster k holds j-tiles
// [cl_jtile[k], cl_jtile[k] + its tile count) and i-records
// [cl_ioff[k], cl_ioff[k] + cl_ni[k]); its active i-particles form
// ceil(cl_ni[k] / i-tile) i-tiles.  A work line lists i-tiles as entries
// {start, cluster, i-tile of the cluster}: entry g covers work positions
// [start_g, start_{g+1}) of the line cut over the CTAs (each position one
// j-tile of the entry's cluster).  hdr[0] = total work W, hdr[1] = number of
// entries n, hdr[2] = index of the line's first entry in gt; entry n (the
// sentinel) has start = W.  Kernels read all of it from device memory, so
// one captured graph serves every step.
struct BatchGT {
    long long start;
    int cluster, itile;
};
struct BatchTables {
    const long long *hdr;
    const BatchGT *gt;
    const int *cl_jtile, *cl_ioff, *cl_ni;
    const double *cl_eps2;
};

// Batch prediction: tile -> cluster map; per cluster first j-tile, particle
// count, active count this step and block time.
struct BatchPredTables {
    const int *tile_cluster, *cl_jtile, *cl_nj, *cl_ni;
    const double *cl_t;
};

// Allocation helpers of the C ABI layer (the device one honours the
// g6x_set_allocator hook; the host one returns mapped pinned memory and its
// device address).
void *dev_alloc_hooked(size_t bytes);
void dev_free_hooked(void *p);
void *host_alloc_zero_copy(size_t bytes, void **dev);
void host_free_pinned(void *p);

// Limit of each bounded wait in the force kernels (nanoseconds); the
// compiled-in value is also the maximum.
void set_wait_limit_ns(unsigned long long ns);
unsigned long long wait_limit_ns();
unsigned long long max_wait_limit_ns();
// One bounded wait that nothing completes; records G6_ETIMEDOUT in *d_err.
cudaError_t launch_wait_probe(int *d_err, cudaStream_t s);

int batch_variant_count();
VariantInfo batch_variant_info(int v);
int batch_variant_occupancy(int v);
cudaError_t launch_predict_batch(int kind, JStore js, Pred p, BatchPredTables bp,
                                 const g6x_jrec *rec, const int *toff, int tile0, int ntiles,
                                 int sm_count, cudaStream_t s);
// tcnt (one zeroed counter per entry of the line, left zeroed): the force
// kernel reduces the entries whose work spans at most FUSED_MAX_SEGS CTAs,
// all with work,
// itself (into out, nearest neighbours mapped through jidx), and the
// reduction launched with fused = true skips them.
cudaError_t launch_force_batch(int v, int grid, const Pred &p, const g6x_irec *d_irec,
                               void *part, int *d_err, const BatchTables &bt, cudaStream_t s,
                               unsigned *tcnt = nullptr, g6x_out *out = nullptr,
                               const int *jidx = nullptr);
cudaError_t launch_reduce_batch(int v, int grid, const void *part, const int *jidx,
                                g6x_out *d_out, const BatchTables &bt, int blocks,
                                cudaStream_t s, bool fused = false);

// The warp-specialised small-block variants (g6gb_small.cu) follow the
// others in one numbering: variant_count() covers both tables.
int variant_count();
VariantInfo variant_info(int v);
int ws_variant_count();
VariantInfo ws_variant_info(int k);
int ws_variant_smem(int k);
int ws_variant_occupancy(int k);
// CTAs per first-level group of the small-block kernel's partial reduction
int ws_group_size(int grid);
// partial records (level 0 and level 1) a small-block launch writes
size_t ws_partial_slots(int grid, int itile);

// Resident CTAs per SM of variant v (0 on error).
int variant_occupancy(int v);
// Pick a variant and grid for ni i-particles against nj_pad j-particles.
// allow_fpred: a fused-prediction shape may be chosen (otherwise its twin).
ForceConfig choose_config(int prec, int ni, int nj_pad, int list, int sm_count,
                          int force_variant, int force_grid, bool allow_fpred = false);
// Whether the built-in choice takes the small-block kernel (where allowed).
extern bool g_ws_default;
// Number of Partial slots a launch with this configuration writes.
size_t partial_slots(const ForceConfig &cfg);
// Ints of list-partial storage a list launch needs with nbseg entries per
// partial: the partials, and for the split-j shapes the runs of their j-groups.
size_t list_part_ints(const ForceConfig &cfg, int nbseg);
// Arrival counters a launch with this configuration needs (zero before it).
size_t counter_slots(const ForceConfig &cfg);

// Autotuning table (see g6x_autotune): per precision and power-of-two
// bucket of ni, the force variant and grid multiplier to use.
constexpr int TUNE_BUCKETS = 32;
int tune_bucket(int ni);
void tune_set(int prec, int bucket, int variant, int gmul);
bool tune_get(int prec, int bucket, int *variant, int *gmul);
bool tune_exact(int prec, int bucket, int *variant, int *gmul);
void tune_clear();

cudaError_t launch_irec_from_store(JStore js, g6x_irec *out, int m, cudaStream_t s);
cudaError_t launch_scatter(const g6x_jrec *d_rec, int n, JStore js,
                           cudaStream_t s);
cudaError_t launch_init_store(JStore js, cudaStream_t s);
// How K1 predicts: the paper's double-single predictor (FP32 Taylor terms
// and a DS + SP addition, Sect. 2.2), the same with the addition done in FP64,
// or everything in FP64 for the FP64 force kernel.
enum PredKind { PRED_DS = 0, PRED_FP64 = 1, PRED_DS_X64 = 2 };
cudaError_t launch_predict(int kind, JStore js, Pred p, int nj, int nj_pad,
                           double t, int sm_count, cudaStream_t s);
// The j-store update fused into the prediction launch: rec holds staged
// records sorted by tile, tile t's at [toff[t], toff[t+1]), for tiles
// 0 .. ntiles_all-1 (which may reach beyond nj_pad / JT).
cudaError_t launch_update_predict(int kind, JStore js, Pred p, int nj, int nj_pad, double t,
                                  const g6x_jrec *rec, const int *toff, int ntiles_all,
                                  int sm_count, cudaStream_t s);
// Neighbour lists of a launch (Sect. 4): maxnb entries kept per i-particle,
// room for nbseg of them per list partial (one CTA's segment of one
// i-particle), and a device int that receives the largest min(count, maxnb)
// of any partial -- above nbseg the lists of that launch are incomplete.
struct ListArgs {
    int maxnb, nbseg;
    int *nbmax;
    // the fused launch also takes the list partials and the output lists
    int *nbl_part = nullptr, *nbc_part = nullptr, *nbl_out = nullptr, *nblen_out = nullptr;
};
cudaError_t launch_force(const ForceConfig &cfg, const Pred &p,
                         const g6x_irec *d_irec, int ni, double eps2,
                         void *part, int *nbl_part, int *nbc_part,
                         int *d_err, cudaStream_t s, const FusedPred *fp = nullptr,
                         bool pdl = false, const ListArgs *lists = nullptr);
// DS force with the reduction fused in: the last CTA to finish an i-tile
// writes its results to out (and with lists, every field of *lists set, the
// concatenated lists).  tcnt holds one counter per i-tile, zero before the
// launch and left zero by a launch that completes.
cudaError_t launch_force_fused(const ForceConfig &cfg, const Pred &p,
                               const g6x_irec *d_irec, int ni, double eps2, void *part,
                               int *d_err, g6x_out *out, const int *jidx, unsigned *tcnt,
                               cudaStream_t s, const FusedPred *fp = nullptr,
                               bool pdl = false, const ListArgs *lists = nullptr);
// One small-block launch (cfg.ws; cfg.grid <= cfg.jtiles, ni <= cfg.itile):
// the j-store update of fp.rec (if any), prediction, force and reduction
// into out; part holds partial_slots(cfg) records, cnt counter_slots(cfg)
// counters, zero before the launch and left zero by a launch that completes.
cudaError_t launch_force_ws(const ForceConfig &cfg, const g6x_irec *d_irec, int ni, double eps2,
                            int nj, void *part, unsigned *cnt, g6x_out *out, const int *jidx,
                            int *d_err, const FusedPred &fp, cudaStream_t s, bool pdl);
cudaError_t launch_reduce(const ForceConfig &cfg, const void *part,
                          const int *nbl_part, const int *nbc_part,
                          const int *jidx, int ni, g6x_out *d_out,
                          int *d_nbl, int *d_nblen, cudaStream_t s, bool pdl = false,
                          const ListArgs *lists = nullptr);
// pdl: launch with programmatic stream serialization (the kernel may start
// behind its predecessor in s and waits for it before reading anything).

}  // namespace g6
