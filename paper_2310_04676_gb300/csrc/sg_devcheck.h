// Device ownership of a context: a context's memory, streams and graphs
// belong to the CUDA device that was current at sg_create, and every entry
// point that touches them checks that this device is current, so that no
// kernel is launched with another device's pointers.
#pragma once

#include <string>

#include "sg.h"

namespace sg {

// owner: the context's device; get_current(int*) -> 0 on success (a
// cudaGetDevice-like query); fn names the entry point in the message.
template <class GetCurrent>
sg_status check_device(int owner, GetCurrent get_current, const char* fn, std::string* msg) {
  int cur = -1;
  if (get_current(&cur) != 0) {
    *msg = std::string(fn) + ": the current CUDA device cannot be queried";
    return SG_ERR_CUDA;
  }
  if (cur != owner) {
    *msg = std::string(fn) + ": the context belongs to CUDA device " + std::to_string(owner) +
           " but device " + std::to_string(cur) +
           " is current; make the context's device current before the call";
    return SG_ERR_INVALID_ARG;
  }
  return SG_OK;
}

}  // namespace sg
