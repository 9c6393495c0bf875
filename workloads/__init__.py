"""Seeded synthetic inputs for the volume/layer-potential evaluator.

This package generates geometry, quadrature nodes and weights, densities and
target points.  It holds none of the evaluation method's arithmetic (no
kernel splitting, no Fourier multipliers, no asymptotics): both the CUDA path
and the CPU oracle consume what it produces, and neither shares any other code.

Modules
-------
curves      closed boundary curves with exact derivatives (circle, ellipse,
            star/starfish r = 1 + a cos k t, the Fourier-coefficient family
            of the paper's numerical section, square)
panels      Gauss-Legendre boundary panels (nodes, weights, outward normals)
quadrature  Gauss-Legendre on [-1,1] and a 6-node degree-4 triangle rule
            obtained by solving its moment equations
mesh        random Delaunay meshes with curved boundary triangles, the
            side-splitting degradation (slivers, hanging nodes, gaps) and a
            jittered structured square mesh
fields      source densities f with analytic derivative jets, smooth
            boundary densities
configs     the concrete workloads (disk, starfish, square, batched star
            domains) and small test problems
"""
