// placeholder translation unit for the tcgen05 GEMMs (filled in below)
