"""GB300 (sm_103a) discrete Frechet distance library.

``paper_2404_05708_gb300.dfd``        -- Python binding of libdfd.so (include/dfd.h)
``paper_2404_05708_gb300.workloads``  -- seeded synthetic inputs (no DFD arithmetic)
``paper_2404_05708_gb300.build``      -- in-tree nvcc build of libdfd.so

Importing the package does not load the CUDA library; ``dfd.load_library``
does, and raises if it is missing.
"""

__all__ = ["dfd", "workloads", "build"]
