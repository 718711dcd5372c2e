// Wavefront transport: queues, counters, BVH queries and the per-path state.
#pragma once

#include "usrt_device.cuh"

namespace usrt {

// path queue, structure of arrays (48 B per path)
struct PathQ {
  float4* pa;   // (o.x, o.y, o.z, a)
  float4* wt;   // (w.x, w.y, w.z, tau_hi)
  uint4* meta;  // (path id, previous primitive code, medium | k << 8, bits(tau_lo))
  float2* surf; // the surface hit carried across a scatterer event: (distance from o, bits(code)),
                // distance < 0 when there is none (the queue the interaction kernel appends to)
  float2* mis;  // with secondary rays at rough events: the direction density of the path's last
                // rough event (0: the last event was not rough) and the distance travelled since
};

// secondary-ray jobs queued by the interaction kernels; round k appends at nee_off[k], so the
// buffer keeps every job of the pass (the adjoint replays them)
// job id word: a scatterer's id, or a triangle's id | NEE_ROUGH for a rough interface event
constexpr uint32_t NEE_ROUGH = 0x80000000u;
struct NeeQ {
  float4* job;      // (a, tau_hi, tau_lo, bits(job id word)) at the event
  uint32_t* jm;     // medium | element << 8 | tx << 16 | k << 24
  uint32_t* jpath;  // path id
  float4* jx;       // rough interface events: (event point, 0)
  float4* jw;       // rough interface events: (incident direction, 0)
};

// what the secondary-ray kernel found for each job, kept for the adjoint of a recorded pass so
// that it need not trace the secondary rays again: per job slot, res = (bits(t_hi), bits(t_lo)
// at the element, gain, sum alpha l) and xo = (first crossing, count), count NEE_NONE for a job
// with no contribution and NEE_UNSTORED when the crossing buffer was full (the adjoint then
// traces that job again); crossings (bits(t), triangle id) in order along the ray.
constexpr uint32_t NEE_NONE = 0xFFFFFFFFu;
constexpr uint32_t NEE_UNSTORED = 0xFFFFFFFEu;
struct NeeRes {
  float4* res;
  uint2* xo;
  uint2* xing;
  uint32_t xcap;
};

// device counters of one transport pass
struct Counters {
  uint32_t live[MAX_KMAX + 2];  // paths entering segment k
  uint32_t nee[MAX_KMAX + 2];   // secondary jobs produced at segment k
  uint32_t nee_off[MAX_KMAX + 2]; // first job of round k in the job buffer
  uint32_t march[MAX_KMAX + 2]; // queue slots claimed by the scatterer march of round k
  uint32_t nee_claim[MAX_KMAX + 2]; // job slots claimed by the secondary-ray kernel of round k
  unsigned long long n_xing;    // secondary-ray crossings appended (NeeRes; may pass xcap)
  uint32_t n_arr;               // arrivals appended
  uint32_t dropped;             // arrivals dropped (crossing list overflow)
  int status;                   // ST_* bits
  uint32_t pad;
};

// arrival: (row = tx * n_elem + e, tq fixed-point time, bits(a), path id)
typedef uint4 Arrival;

// coherence sort of a ray queue: one counting-sort pass over a 14-bit key (origin cell in x and
// z, octahedral direction bin), so that the lanes of a warp start near each other and point the
// same way.  Rays that carry their surface hit across a scatterer event (a pass-through: the
// surface ahead is the one already found) follow in RAY_CARRY_BUCKETS coarser buckets of their
// own, so the surface query runs over the first RAY_KEY_BUCKETS buckets only.  The kernel that
// appends a ray to the queue (emission, interaction) writes its key and counts it, so the sort
// itself is the scan of the counts and one scatter pass.
constexpr int RAY_KEY_BITS = 14;
constexpr int RAY_KEY_BUCKETS = 1 << RAY_KEY_BITS;
constexpr int RAY_CARRY_BUCKETS = 1024;
constexpr int RAY_BUCKETS = RAY_KEY_BUCKETS + RAY_CARRY_BUCKETS;
struct RaySort {
  float3 lo, inv_ext;   // scene bounds for the origin cells
  uint32_t* key;        // per ray
  uint32_t* cnt;        // [RAY_BUCKETS]
  uint32_t* off;        // [RAY_BUCKETS + 1]
  uint32_t* cursor;     // [RAY_BUCKETS]
};

struct TransportArgs {
  SceneDev S;
  Media med;
  Acq acq;
  PathQ qin, qout;
  float2* hits;       // (t, bits(code)) per queue slot
  float2* keep;       // per queue slot: the surface hit a scatterer event replaced in hits
  const uint32_t* trav_n;  // rays of the sorted queue that need a surface query (the rest carry one)
  RaySort rk;         // keys and bucket counts of the rays appended to qout (the next round's sort)
  bool mis_on;        // secondary rays at rough events (the queues' mis fields are live)
  NeeQ nee;
  NeeRes nres;        // null members unless the pass is recorded for the adjoint
  Arrival* arr;       // may be null (adjoint recompute: no arrivals)
  uint32_t arr_cap;
  uint32_t* record;   // may be null; index (path - path_base) * (kmax + 1) + k
  long long path_base;
  Counters* cnt;
  int k;              // segment index
};

// sorts queue `from` (count live[k]; its keys and counts written by the kernel that filled it,
// into the counts zeroed before that kernel) into `to`
void launch_ray_sort(const TransportArgs& a, const PathQ& from, const PathQ& to, const RaySort& rs, int grid,
                     cudaStream_t st);
// sorts round k's secondary-ray jobs (from.[nee_off[k], + nee[k])) into the same range of `to`
// by target element and origin cell: jobs aimed at one element from nearby scatterers share a
// warp
void launch_job_sort(const TransportArgs& a, const NeeQ& from, const NeeQ& to, const RaySort& rs, int grid,
                     cudaStream_t st);
cudaError_t ray_sort_set_attrs();

// emission of paths [path0, path0 + n) straight into coherence-sorted order in a.qout (its keys
// counted into rs.cnt, zeroed by the caller, then scanned)
void launch_generate(const TransportArgs& a, long long path0, uint32_t n, const RaySort& rs, int grid,
                     cudaStream_t st);
constexpr int TRAV_THREADS = 128;
void launch_traverse(const TransportArgs& a, int grid, cudaStream_t st);
int traverse_blocks_per_sm();  // blocks per SM of the traversal grid
constexpr int MARCH_THREADS = 128;
void launch_march(const TransportArgs& a, int grid, cudaStream_t st);
int march_blocks_per_sm();  // resident blocks per SM of the scatterer march (persistent grid)
void launch_interact(const TransportArgs& a, int grid, cudaStream_t st);
constexpr int NEE_THREADS = 128;
void launch_nee(const TransportArgs& a, int grid, cudaStream_t st);
int nee_blocks_per_sm();  // resident blocks per SM of the secondary-ray kernel (persistent grid)

}  // namespace usrt
