// Shared declarations of the batched (many fields, one pass) search.
#pragma once

#include "sas_internal.cuh"

namespace sas {

// Per-field 32-bit counters (one row of kCtrN words per field).
enum : int {
  kCtrFlags = 0,  // error / capacity flags of the field
  kCtrEmit = 1,   // emitted super-bins
  kCtrValid = 2,  // bins with >= n_min distinct epochs
  kCtrOut = 3,    // candidates kept (after the optional top-K cut)
  kCtrIdsLo = 4,  // total contributing ids (low / high word)
  kCtrIdsHi = 5,
  kCtrN = 8
};
// Per-field 64-bit counters.
enum : int { kC64Pairs = 0, kC64Balance = 1, kC64T0 = 2, kC64N = 4 };

// Initial candidate-key slots of one field (a power of two: every field's keys
// form one segment of a segmented sort); a batch whose fields need more grows
// its segment to the next power of two and rebuilds its pass.
constexpr uint32_t kBatchKeyCap = 32768;
constexpr uint32_t kBatchKeyCapMax = 1u << 22;

// Everything the batch kernels need to know about one field.
struct BatchField {
  StackArgs args;             // stack kernel arguments (pointers into the batch arena)
  const int32_t* x;           // caller's catalog (device)
  const int32_t* y;
  const uint16_t* epoch;
  const int64_t* t;           // epoch times (device copy)
  uint32_t E;
  uint32_t emit_cap;
  uint32_t* ecount;           // [E]
  int64_t* dt;                // [E]
  long long* t0;              // -> this field's kC64T0 counter
  int32_t* sxt;               // [nvx][E]
  int32_t* syt;               // [nvy][E]
  uint64_t bucket_base;       // first bucket of the field in the global bucket arrays
  uint32_t* counters;         // [kCtrN]
  Key* keys;                  // [key_cap]
  uint32_t key_cap;
  uint32_t max_out;           // top-K cut
  unsigned long long* id_off; // [key_cap + 1]
  uint32_t* ids;              // [ids_cap]
  uint32_t* ids_tmp;          // [ids_cap]
  uint64_t ids_cap;
  sas_candidate* cands;       // [key_cap]
};

// Device views of a batch and its totals (host struct passed to the launchers).
struct BatchDev {
  BatchField* fields;
  int n_fields;
  unsigned long long* det_off;   // [n_fields + 1] detections
  unsigned long long total_dets;
  uint32_t* bucket_count;
  uint32_t* boff;                // [total_buckets + 1]
  uint32_t* cursor;
  uint32_t* scan_scratch;
  uint64_t total_buckets;
  uint32_t* bucket_of;           // [total_dets]
  Det* dets;                     // [total_dets]
  unsigned long long* tab_off;   // [n_fields + 1] shift-table entries (x then y)
  unsigned long long total_tab;
  unsigned long long* emit_off;  // [n_fields + 1] emission slots
  unsigned long long total_emit;
  unsigned long long* cand_off;  // [n_fields + 1] candidate slots
  unsigned long long total_cand;
  uint32_t key_seg;              // key slots per field (a power of two)
  Key* keys_all;                 // [total_cand]: field f's keys at cand_off[f]
};

cudaError_t batch_launch_prep(const BatchDev& B, cudaStream_t s);
cudaError_t batch_launch_post(const BatchDev& B, cudaStream_t s);
cudaError_t batch_set_attrs();

// Vetting of a batch (sas_batch_vet): ownership selection of every active
// field's candidates in one pass over the arena.  active[f] != 0 for fields whose
// results are in the arena; owner has total_dets words (all 0xFFFFFFFF on entry),
// flag total_cand words (all 0 on entry).  Then the in-order compaction of the
// flags into (field, candidate) pairs.
cudaError_t batch_launch_owned(const BatchDev& B, const uint8_t* active, uint32_t* owner, uint32_t* flag,
                               cudaStream_t s);
cudaError_t batch_launch_compact(const BatchDev& B, const uint32_t* flag, const uint32_t* off,
                                 uint32_t* field_out, uint32_t* cand_out, cudaStream_t s);
// Stamps of (field[i], cand[i]) pairs (sas_stamps.cu); max_e: largest epoch count.
cudaError_t launch_batch_stamps(const BatchField* F, uint32_t max_e, const uint32_t* field, const uint32_t* cand,
                                uint64_t n, uint16_t* out, cudaStream_t s);

}  // namespace sas
