#!/bin/bash
# DRAM traffic of the benchmark's render launch for every kernel variant (one-pass ncu metrics), as recorded in
# measured_traffic.json.  Run from the repository root on a GPU machine; each variant's plain run comes first.
set -e
out=${1:-traffic}
mkdir -p "$out"
n=$(python -c "from paper_2011_03082_b300 import ms; print(ms.lib().ms_render_variants())")
for v in $(seq 0 $((n - 1))); do
  python bench.py --steps 1 --warmup 3 --no-cpu --no-equal-rmse --no-brute --variant "$v" > "$out/plain_$v.log" 2>&1
  ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none \
      -k regex:render_kernel --csv --log-file "$out/dram_$v.csv" \
      python bench.py --steps 1 --warmup 3 --no-cpu --no-equal-rmse --no-brute --variant "$v" > "$out/ncu_$v.log" 2>&1
done
