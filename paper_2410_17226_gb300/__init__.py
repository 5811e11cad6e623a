"""GB300-native Cluster-BFS (arXiv 2410.17226): CUDA kernels behind a C ABI.

``cbfs``   -- the Python binding of libcbfs.so (Graph, Labels, run, query);
``inputs`` -- seeded synthetic graphs and clusters;
``serve``  -- continuous-batching distance-query server over device labels;
``tune``   -- autotuner for the traversal's push/pull switch and slot count;
``build``  -- compiles libcbfs.so for sm_103a.
"""
