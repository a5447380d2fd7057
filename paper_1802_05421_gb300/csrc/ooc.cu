// Chain levels kept in pinned host memory (the larger-than-memory form: the
// paper's larger-than-memory aim; here the host holds the levels and the GPU
// streams them). The first `resident` levels may stay in device memory (a
// chain larger than the host's memory keeps what fits on the device); the
// rest live on the host. Two device slots hold the host levels in use. A
// squaring reads level i from one slot (or from device memory) and writes
// level i + 1 into the other, which is then copied out to the host on a copy
// stream while the next squaring runs; an application of the chain loads
// level l + 1 into the free slot while level l is applied. Events order every
// slot reuse: a slot is overwritten only after its previous level has been
// copied out and its last reader has finished.
#include <algorithm>

#include "internal.h"

namespace cdl {

namespace {
size_t level_bytes(const cdl_chain* ch) { return (size_t)ch->npad * (size_t)ch->npad * 2; }

bool resident(const cdl_chain* ch, int i) { return i < ch->resident; }
void* dev_level(const cdl_chain* ch, int i) { return static_cast<char*>(ch->dev_levels) + (size_t)i * level_bytes(ch); }
void* host_level(const cdl_chain* ch, int i) {
  return static_cast<char*>(ch->levels) + (size_t)(i - ch->resident) * level_bytes(ch);
}

int slot_holding(const cdl_chain* ch, int i) {
  for (int s = 0; s < 2; ++s)
    if (ch->slot_level[s] == i) return s;
  return -1;
}

// the slot a new level may go to: not the one holding the level used last
int victim(const cdl_chain* ch) {
  if (ch->last_level < 0) return 0;
  return ch->slot_level[0] == ch->last_level ? 1 : 0;
}

// issue the load of level i into slot s on the copy stream
int load(cdl_ctx* ctx, cdl_chain* ch, int i, int s) {
  CDL_CUDA_TRY(cudaStreamWaitEvent(ch->copy, ch->ev_free[s], 0));
  CopyTimer T(ctx, ch->copy, (double)level_bytes(ch));
  CDL_CUDA_TRY(cudaMemcpyAsync(ch->slot[s], host_level(ch, i), level_bytes(ch), cudaMemcpyHostToDevice, ch->copy));
  T.done();
  CDL_CUDA_TRY(cudaEventRecord(ch->ev_ready[s], ch->copy));
  ch->slot_level[s] = i;
  ch->link_bytes += (double)level_bytes(ch);
  return CDL_OK;
}
}  // namespace

int ooc_init(cdl_chain* ch) {
  const size_t lb = level_bytes(ch);
  ch->resident = std::min(ch->resident, ch->d);
  if (ch->resident > 0 && cudaMalloc(&ch->dev_levels, (size_t)ch->resident * lb) != cudaSuccess) {
    cudaGetLastError();
    ch->dev_levels = nullptr;
    return CDL_ERR_OOM;
  }
  if (ch->resident == ch->d) {   // nothing on the host: no slots, no copies
    ch->host_levels = true;
    return CDL_OK;
  }
  if (cudaHostAlloc(&ch->levels, (size_t)(ch->d - ch->resident) * lb, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    ch->levels = nullptr;
    return CDL_ERR_OOM;
  }
  for (int s = 0; s < 2; ++s) {
    if (cudaMalloc(&ch->slot[s], lb) != cudaSuccess || cudaEventCreateWithFlags(&ch->ev_ready[s], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ch->ev_free[s], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return CDL_ERR_OOM;
    }
  }
  if (cudaStreamCreateWithFlags(&ch->copy, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return CDL_ERR_CUDA;
  }
  ch->host_levels = true;
  return CDL_OK;
}

void ooc_destroy(cdl_chain* ch) {
  if (ch->copy) cudaStreamSynchronize(ch->copy);
  for (int s = 0; s < 2; ++s) {
    if (ch->slot[s]) cudaFree(ch->slot[s]);
    if (ch->ev_ready[s]) cudaEventDestroy(ch->ev_ready[s]);
    if (ch->ev_free[s]) cudaEventDestroy(ch->ev_free[s]);
    ch->slot[s] = nullptr;
  }
  if (ch->copy) cudaStreamDestroy(ch->copy);
  ch->copy = nullptr;
  if (ch->levels) cudaFreeHost(ch->levels);
  ch->levels = nullptr;
  if (ch->dev_levels) cudaFree(ch->dev_levels);
  ch->dev_levels = nullptr;
}

void* ooc_level_ptr(const cdl_chain* ch, int i) { return resident(ch, i) ? dev_level(ch, i) : host_level(ch, i); }

void* ooc_write_begin(cdl_ctx* ctx, cdl_chain* ch, int i) {
  if (resident(ch, i)) return dev_level(ch, i);   // ordered on the stream like any device level
  int s = slot_holding(ch, i);
  if (s < 0) s = victim(ch);
  cudaStreamWaitEvent(ctx->stream, ch->ev_free[s], 0);    // old level saved / read
  cudaStreamWaitEvent(ctx->stream, ch->ev_ready[s], 0);   // and no load into the slot still in flight
  ch->slot_level[s] = i;                                  // (a prefetch may have started one, e.g. of
  return ch->slot[s];                                     // level 0 of the previous graph's chain)
}

int ooc_write_end(cdl_ctx* ctx, cdl_chain* ch, int i) {
  if (resident(ch, i)) return CDL_OK;
  const int s = slot_holding(ch, i);
  if (s < 0) return CDL_ERR_INVALID_ARG;
  CDL_CUDA_TRY(cudaEventRecord(ch->ev_ready[s], ctx->stream));
  CDL_CUDA_TRY(cudaStreamWaitEvent(ch->copy, ch->ev_ready[s], 0));
  CopyTimer T(ctx, ch->copy, (double)level_bytes(ch));
  CDL_CUDA_TRY(cudaMemcpyAsync(host_level(ch, i), ch->slot[s], level_bytes(ch), cudaMemcpyDeviceToHost, ch->copy));
  T.done();
  CDL_CUDA_TRY(cudaEventRecord(ch->ev_free[s], ch->copy));
  ch->link_bytes += (double)level_bytes(ch);
  ch->last_level = i;
  return CDL_OK;
}

const void* ooc_read(cdl_ctx* ctx, cdl_chain* ch, int i) {
  if (resident(ch, i)) return dev_level(ch, i);
  int s = slot_holding(ch, i);
  if (s < 0) {
    s = victim(ch);
    if (load(ctx, ch, i, s) != CDL_OK) return nullptr;
  }
  if (cudaStreamWaitEvent(ctx->stream, ch->ev_ready[s], 0) != cudaSuccess) return nullptr;
  return ch->slot[s];
}

int ooc_read_done(cdl_ctx* ctx, cdl_chain* ch, int i) {
  if (resident(ch, i)) return CDL_OK;
  const int s = slot_holding(ch, i);
  if (s < 0) return CDL_ERR_INVALID_ARG;
  CDL_CUDA_TRY(cudaEventRecord(ch->ev_free[s], ctx->stream));
  ch->last_level = i;
  return CDL_OK;
}

// Issued after ooc_read_done of the level in use, so a load into its slot
// (a chain of one level) waits for that reader.
int ooc_prefetch(cdl_ctx* ctx, cdl_chain* ch, int i) {
  if (resident(ch, i) || slot_holding(ch, i) >= 0) return CDL_OK;
  return load(ctx, ch, i, victim(ch));
}

}  // namespace cdl
