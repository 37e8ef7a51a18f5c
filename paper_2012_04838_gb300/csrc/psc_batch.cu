// Host side of the persistent ensemble kernel (psc_batch_kernel.cuh): the
// work table's layout and construction, and the captured step of four
// per-stage launches (psc_batch_stage.cu, one unit per stage).
#include "psc_batch_kernel.cuh"

#define PSCB_DECL(s)                                                                                      \
  cudaError_t pscb_launch_stage_##s(bool big, int grid, size_t smem, cudaStream_t st, const void* head,  \
                                    const void* boxes, const void* segs, void* counters);                \
  int pscb_prepare_stage_##s(bool big, size_t smem);
PSCB_DECL(1)
PSCB_DECL(2)
PSCB_DECL(3)
PSCB_DECL(4)
#undef PSCB_DECL

// ---------------------------------------------------------------- host side

bool pscb_size_supported(int N) {
  switch (N) {
#define PSCB_S(n) case n: return true;
    PSCB_SIZES(PSCB_S)
#undef PSCB_S
    default: return false;
  }
}

size_t pscb_smem_bytes(int max_N) {
  size_t m = 0;
#define PSCB_M(n) if (n <= max_N && smem_of<n>() > m) m = smem_of<n>();
  PSCB_SIZES(PSCB_M)
#undef PSCB_M
  return m;
}

size_t pscb_table_bytes(int max_boxes) { return table_layout(max_boxes).total; }

cudaError_t pscb_upload(void* table, void* staging, int max_boxes, const PscBatchBox* boxes, int n,
                        cudaStream_t st, bool stall_test) {
  const TableLayout L = table_layout(max_boxes);
  unsigned char* h = static_cast<unsigned char*>(staging);
  std::memset(h, 0, L.counters);
  Head* hd = reinterpret_cast<Head*>(h + L.head);
  hd->nbox = n;
  hd->wait_ns = stall_test ? kStallTestWaitNs : kWaitNs;
  if (n > 0) std::memcpy(h + L.boxes, boxes, sizeof(PscBatchBox) * (size_t)n);
  for (int stage = 1; stage <= 4; ++stage) {
    Seg* sg = reinterpret_cast<Seg*>(h + L.segs) + (size_t)(stage - 1) * L.seg_cap;
    int ns = 0;
    long long off = 0;
    std::vector<int> last(n, -1), last_tiles(n, 0);
    for (int p = 0; p < BP_N; ++p) {
      for (int bi = 0; bi < n; ++bi) {
        const int t = tiles_dispatch(boxes[bi].N, p, stage, boxes[bi]);
        if (t <= 0) continue;
        Seg& s = sg[ns++];
        s.start = off;
        s.box = bi;
        s.pass = p;
        s.tiles = t;
        s.per = tiles_per_item(p);
        const int items = (t + s.per - 1) / s.per;
        s.dep = last[bi];
        s.dep_tiles = last_tiles[bi];
        s.done_idx = bi * BP_N + p;
        last[bi] = s.done_idx;
        last_tiles[bi] = items;  // done[] counts items
        off += items;
      }
    }
    hd->nseg[stage - 1] = ns;
    hd->nitems[stage - 1] = off;
    if (stall_test && stage == 1) {
      // failure-path test: the first item that waits at stage 1 waits for one
      // tile more than its dependency has, so its bounded wait runs out
      for (int i = 0; i < ns; ++i)
        if (sg[i].dep >= 0) {
          sg[i].dep_tiles += 1;
          break;
        }
    }
  }
  return cudaMemcpyAsync(table, staging, L.counters, cudaMemcpyHostToDevice, st);
}

int pscb_grid(int max_N, size_t smem) {
  const bool big = max_N > 128;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per = pscb_prepare_stage_1(big, smem);
  const int p2 = pscb_prepare_stage_2(big, smem), p3 = pscb_prepare_stage_3(big, smem),
            p4 = pscb_prepare_stage_4(big, smem);
  per = per < p2 ? per : p2;
  per = per < p3 ? per : p3;
  per = per < p4 ? per : p4;
  if (per < 1) per = 1;
  return (sms > 0 ? sms : 152) * per;
}

cudaError_t pscb_step(void* table, int max_boxes, int max_N, int grid, size_t smem, cudaStream_t st) {
  const bool big = max_N > 128;
  const TableLayout L = table_layout(max_boxes);
  unsigned char* t = static_cast<unsigned char*>(table);
  cudaError_t e = cudaMemsetAsync(t + L.counters, 0, 4 * L.counter_bytes, st);
  if (e != cudaSuccess) return e;
  const void* head = t + L.head;
  const void* boxes = t + L.boxes;
  const Seg* segs = reinterpret_cast<const Seg*>(t + L.segs);
  e = pscb_launch_stage_1(big, grid, smem, st, head, boxes, segs, t + L.counters);
  if (e == cudaSuccess)
    e = pscb_launch_stage_2(big, grid, smem, st, head, boxes, segs + L.seg_cap, t + L.counters + L.counter_bytes);
  if (e == cudaSuccess)
    e = pscb_launch_stage_3(big, grid, smem, st, head, boxes, segs + 2 * L.seg_cap,
                            t + L.counters + 2 * L.counter_bytes);
  if (e == cudaSuccess)
    e = pscb_launch_stage_4(big, grid, smem, st, head, boxes, segs + 3 * L.seg_cap,
                            t + L.counters + 3 * L.counter_bytes);
  return e;
}
