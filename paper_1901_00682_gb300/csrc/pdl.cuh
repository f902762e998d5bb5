// Programmatic dependent launch: a kernel launched with the programmatic stream
// serialisation attribute may start while the kernel before it in the stream is still
// running.  griddep_wait() returns once that kernel has completed and its memory
// writes are visible (at once when there is no such kernel or the attribute is off), so
// every access to data the previous kernel writes, or reads and this one overwrites,
// comes after it.  griddep_launch() lets the next kernel of the stream, if it was
// launched with the attribute, start once every CTA of this grid has called it or
// exited; its own griddep_wait() still waits for this grid's completion.
#pragma once

#include <cuda_runtime.h>

namespace ddtv {

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// appends the attribute to a launch configuration whose attrs array has a free slot
inline void allow_programmatic_launch(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attrs) {
  attrs[cfg.numAttrs].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attrs[cfg.numAttrs].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attrs;
  ++cfg.numAttrs;
}

}  // namespace ddtv
