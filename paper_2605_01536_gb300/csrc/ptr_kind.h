// Classification of a caller's buffer for a launch on one device, from the
// attributes the CUDA runtime reports for it (host code, no CUDA calls).
#pragma once

// type: the cudaMemoryType value (0 unregistered, 1 host, 2 device, 3 managed);
// ptr_device: the device the runtime names for the buffer; device: the device
// the kernels will run on.  Returns 1 if the kernels may read the buffer in
// place (device memory of `device`, or managed memory), 0 for host memory
// (staged through the device by the callers that accept it), -1 for device
// memory of another GPU, which is refused: a kernel on `device` that
// dereferenced it would fault.
static inline int gwn_pointer_kind_of(int type, int ptr_device, int device) {
    if (type == 3) return 1;
    if (type == 2) return ptr_device == device ? 1 : -1;
    return 0;
}
